"""A failed host allocation inside the set-up ends as SEIRD_ENOMEM with a
message, never as an exception crossing the C ABI (which would abort the
process).  The child process caps its own address space just above what it
already maps, so the set-up's host arrays cannot be allocated; the worker
threads of the set-up cannot start either and the calling thread works alone.
No GPU: the set-up runs before any device call."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import resource, sys
    sys.path.insert(0, {root!r})
    from paper_2208_01839_gb300 import inputs as I
    from paper_2208_01839_gb300 import seird as S

    xy, tri = I.structured_mesh(600)
    params = I.params_square()
    for _ in range(2):  # the first calls map what the library and the allocator keep
        S.setup_check(xy, tri, n_subdomains=64, overlap=2)
    vm = [int(l.split()[1]) for l in open("/proc/self/status") if l.startswith("VmSize")][0] * 1024
    cap = vm + (32 << 20)
    resource.setrlimit(resource.RLIMIT_AS, (cap, cap))
    for call in (lambda: S.setup_check(xy, tri, n_subdomains=64, overlap=2),
                 lambda: S.Solver(xy, tri, params, n_subdomains=64, overlap=2)):
        try:
            call()
        except S.SeirdError as e:
            print("code", e.code, str(e))
        else:
            print("no error")
""")


@pytest.mark.skipif(not sys.platform.startswith("linux"), reason="uses /proc and RLIMIT_AS")
def test_failed_host_allocation_is_an_error_code():
    from paper_2208_01839_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    lines = [l for l in r.stdout.splitlines() if l.startswith("code") or l == "no error"]
    assert len(lines) == 2, r.stdout
    for l in lines:
        assert l.startswith("code -2") and "host allocation failed" in l, l
