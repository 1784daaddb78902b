"""swpic_deposit_static: the deposit for callers that cannot let the library
allocate device memory (its scratch is a fixed file-scope device array).

Checked through the C ABI against the regular path (swpic_deposit, then the
b of swpic_get_mesh) on the same particles, within the deposit tolerance of
the other tests (1e-5 relative for FP32 states, 1e-12 for FP64), on two calls
in a row with different particles, so a second call must not see the first
call's charge; and against the FP64 oracle's deposit (Eq. rhs-assembly) of
the same stored values.  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import cast_state, need_gpu, rel_max

pytestmark = pytest.mark.gpu


def _static(torch, swpic, st, prec, L, nx, stream, decorated=True):
    dt = torch.float32 if prec == 32 else torch.float64
    dev = {k: torch.from_numpy(st[k]).to(device="cuda", dtype=dt) for k in ("Q", "ps", "psi")}
    b = torch.full((nx,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    lib = swpic.load_library()
    st_ = lib.swpic_deposit_static(dev["Q"].data_ptr(), dev["ps"].data_ptr() if decorated else None,
                                   dev["psi"].data_ptr(), len(st["Q"]), prec, L, nx, b.data_ptr(),
                                   stream.cuda_stream)
    stream.synchronize()
    return st_, b.cpu().numpy()


def _context_b(swpic, st, prec, L, nx, decorated=True):
    n = len(st["Q"])
    sim = swpic.Simulation([(L, 0.1, nx, n)], precision=prec, decorated=decorated)
    try:
        sim.init_particles(st)
        swpic.swpic_deposit(sim.ctx)
        return sim.mesh(0)["b"]
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_static_deposit_matches_context_deposit_twice(prec):
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    L, nx = 4 * np.pi, 512
    tol = 1e-5 if prec == 32 else 1e-12
    stream = torch.cuda.Stream()
    for call, (n, seed) in enumerate(((200003, 7), (65536, 8))):
        st = W.random_state(n, L, seed=seed, nx=nx)
        ref = _context_b(swpic, st, prec, L, nx)
        rc, got = _static(torch, swpic, st, prec, L, nx, stream)
        assert rc == swpic.SWPIC_OK
        assert np.all(np.isfinite(got)), call
        assert rel_max(got, ref) <= tol, (call, rel_max(got, ref))
        s = cast_state(st, prec)
        orc = O.deposit(s["Q"], s["ps"], s["psi"], L, nx)
        assert rel_max(got, orc) <= tol, (call, rel_max(got, orc))


@pytest.mark.parametrize("prec", [32, 64])
def test_static_deposit_wraps_positions_outside_the_domain(prec):
    """Positions just below 0, exactly L and beyond L are wrapped into [0, L)
    as the context path wraps them, so both give the same b."""
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    L, nx = 4 * np.pi, 64
    h = L / nx
    st = W.random_state(4099, L, seed=3, nx=nx)
    st["Q"][:6] = [-0.1 * h, L, L + 0.3 * h, -L - 0.2 * h, 3 * L + 0.7 * h, -2.5 * L]
    ref = _context_b(swpic, st, prec, L, nx)
    rc, got = _static(torch, swpic, st, prec, L, nx, torch.cuda.Stream())
    assert rc == swpic.SWPIC_OK
    tol = 1e-5 if prec == 32 else 1e-12
    assert rel_max(got, ref) <= tol, rel_max(got, ref)


def test_static_deposit_largest_mesh_and_no_decoration():
    """nx = SWPIC_STATIC_NX_MAX (the node j = nx folds into node 0 at the
    largest shared tile) matches the context path, with and without p*."""
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    L, nx = 20.0, swpic.SWPIC_STATIC_NX_MAX
    st = W.random_state(300001, L, seed=11, nx=nx)
    stream = torch.cuda.Stream()
    for dec in (True, False):
        ref = _context_b(swpic, st, 32, L, nx, decorated=dec)
        rc, got = _static(torch, swpic, st, 32, L, nx, stream, decorated=dec)
        assert rc == swpic.SWPIC_OK
        assert rel_max(got, ref) <= 1e-5, (dec, rel_max(got, ref))


def test_static_deposit_rejects_meshes_beyond_its_scratch():
    torch = need_gpu()
    from paper_2605_21794_gb300 import swpic
    lib = swpic.load_library()
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    q = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = lib.swpic_deposit_static(q.data_ptr(), None, q.data_ptr(), 4, 32, 1.0,
                                  swpic.SWPIC_STATIC_NX_MAX + 1, b.data_ptr(), None)
    assert st == swpic.SWPIC_EINVAL
