"""swpic_deposit_static: the deposit for callers that cannot let the library
allocate device memory (its scratch is a fixed file-scope device array).

Checked through the C ABI against the regular path (swpic_deposit, then the
b of swpic_get_mesh) on the same particles, within the deposit tolerance of
the other tests (1e-5 relative for FP32 states, 1e-12 for FP64), on two calls
in a row with different particles, so a second call must not see the first
call's charge.  Collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_gpu, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [32, 64])
def test_static_deposit_matches_context_deposit_twice(prec):
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    L, nx = 4 * np.pi, 512
    tol = 1e-5 if prec == 32 else 1e-12
    dt = torch.float32 if prec == 32 else torch.float64
    stream = torch.cuda.Stream()
    for call, (n, seed) in enumerate(((200003, 7), (65536, 8))):
        st = W.random_state(n, L, seed=seed, nx=nx)
        sim = swpic.Simulation([(L, 0.1, nx, n)], precision=prec)
        try:
            sim.init_particles(st)
            swpic.swpic_deposit(sim.ctx)
            ref = sim.mesh(0)["b"]
            dev = {k: torch.from_numpy(st[k]).to(device="cuda", dtype=dt) for k in ("Q", "ps", "psi")}
            b = torch.full((nx,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            swpic.swpic_deposit_static(dev["Q"].data_ptr(), dev["ps"].data_ptr(), dev["psi"].data_ptr(),
                                       n, prec, L, nx, b.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            got = b.cpu().numpy()
        finally:
            sim.close()
        assert np.all(np.isfinite(got)), call
        assert rel_max(got, ref) <= tol, (call, rel_max(got, ref))


def test_static_deposit_rejects_meshes_beyond_its_scratch():
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    lib = swpic.load_library()
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    q = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = lib.swpic_deposit_static(q.data_ptr(), None, q.data_ptr(), 4, 32, 1.0,
                                  swpic.SWPIC_NX_MAX + 1, b.data_ptr(), None)
    assert st == swpic.SWPIC_EINVAL
