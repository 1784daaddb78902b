"""GPU parity of the decorated-particle initialization from marker particles
(Sec. 4.1-4.2, Alg. lumping_procedure) against the oracle, through the C ABI.

Both sides take the nearest-center decision in FP32 from the same separately
rounded operations; the GPU's member sums are exact (fixed point) and the
oracle's are sequential FP64, so the FP32-rounded centers agree unless a
mean sits within ~1e-8 of a float rounding boundary, which these seeded
inputs avoid.  Hence: assignments bit-exact, the chosen central markers
(Q, P) bit-exact, centers / psi* / p* / q* within 1e-12 (FP64 summation
order).  At the full size (1e5 markers, 1e4 clusters, the oracle too slow)
the torus moment requirements are checked per cluster instead.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu
L = 2 * np.pi


def _dev(a, torch, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype or torch.float64)


def _gpu_kmeans(m, cq0, cp0, n_iter):
    import torch
    from paper_2605_21794_gb300 import swpic
    M, K = len(m["Q"]), len(cq0)
    Qm, Pm, wm = _dev(m["Q"], torch), _dev(m["P"], torch), _dev(m["psi"], torch)
    cq, cp = _dev(cq0, torch), _dev(cp0, torch)
    assign = torch.zeros(max(M, 1), dtype=torch.int32, device="cuda")
    out = [torch.zeros(K, dtype=torch.float64, device="cuda") for _ in range(5)]
    stream = torch.cuda.current_stream().cuda_stream
    n = swpic.swpic_kmeans_lump(Qm.data_ptr(), Pm.data_ptr(), wm.data_ptr(), M, cq.data_ptr(), cp.data_ptr(),
                                K, L, n_iter, assign.data_ptr(), *[o.data_ptr() for o in out], stream)
    Q, P, qs, ps, psi = [o.cpu().numpy()[:n] for o in out]
    return {"cq": cq.cpu().numpy(), "cp": cp.cpu().numpy(), "assign": assign.cpu().numpy()[:M],
            "Q": Q, "P": P, "qs": qs, "ps": ps, "psi": psi}


def _per_d(a, b):
    d = a - b
    return d - L * np.round(d / L)


@pytest.mark.parametrize("M,K,n_iter,seed", [(20000, 1000, 8, 1), (6001, 317, 5, 2), (5000, 1, 3, 3)])
def test_kmeans_lump_matches_oracle(M, K, n_iter, seed):
    need_gpu()
    m = W.two_stream_markers(M, seed)
    cq0, cp0 = m["Q"][:K].copy(), m["P"][:K].copy()
    got = _gpu_kmeans(m, cq0, cp0, n_iter)
    cq, cp, a = O.kmeans(m["Q"], m["P"], m["psi"], cq0, cp0, L, n_iter)
    ref = O.lump(m["Q"], m["P"], m["psi"], a, cq, cp, L)
    assert np.array_equal(got["assign"], a)
    assert np.abs(_per_d(got["cq"], cq)).max() <= 1e-12
    assert np.abs(got["cp"] - cp).max() <= 1e-12
    assert len(got["Q"]) == len(ref["Q"])
    assert np.array_equal(got["Q"], ref["Q"]) and np.array_equal(got["P"], ref["P"])
    assert np.abs(got["psi"] - ref["psi"]).max() <= 1e-13 * ref["psi"].max()
    scale = ref["psi"].max()
    assert np.abs(got["ps"] - ref["ps"]).max() <= 1e-12 * scale
    assert np.abs(got["qs"] - ref["qs"]).max() <= 1e-12 * scale


def test_empty_clusters_are_skipped_and_calls_repeat_bitwise():
    need_gpu()
    m = W.two_stream_markers(3000, 4)
    K = 64
    cq0 = np.concatenate([m["Q"][:32], np.full(32, 1.0)])
    cp0 = np.concatenate([m["P"][:32], np.full(32, 50.0)])        # far from every marker: stay empty
    g1 = _gpu_kmeans(m, cq0, cp0, 4)
    g2 = _gpu_kmeans(m, cq0, cp0, 4)
    cq, cp, a = O.kmeans(m["Q"], m["P"], m["psi"], cq0, cp0, L, 4)
    ref = O.lump(m["Q"], m["P"], m["psi"], a, cq, cp, L)
    assert len(g1["Q"]) == len(ref["Q"]) <= 32
    assert np.array_equal(g1["assign"], a)
    for k in ("assign", "cq", "cp", "Q", "P", "psi"):
        assert np.array_equal(g1[k], g2[k]), k
    assert np.all(g1["cp"][32:] == 50.0)                          # empty clusters keep their centers


def test_full_size_moment_requirements():
    """1e5 markers of the two-stream sample, 1e4 clusters: per cluster the
    decorated particle reproduces the markers' sin(2 pi (q - Q)/L) and p
    moments (the torus requirements), psi* conserves the weight, and every
    assignment is a nearest final center within FP32 rounding."""
    need_gpu()
    M, K = 100000, 10000
    m = W.two_stream_markers(M, 7)
    g = _gpu_kmeans(m, m["Q"][:K].copy(), m["P"][:K].copy(), 10)
    a = g["assign"]
    ks = np.unique(a)
    assert len(g["Q"]) == len(ks)
    assert g["psi"].sum() == pytest.approx(m["psi"].sum(), rel=1e-13)
    w = m["psi"]
    sin_m = np.bincount(a, weights=w * np.sin(2 * np.pi * (m["Q"] - g["Q"][np.searchsorted(ks, a)]) / L),
                        minlength=K)[ks]
    assert np.allclose(sin_m, -g["ps"] * 2 * np.pi / L, atol=1e-13, rtol=0)
    p_m = np.bincount(a, weights=w * m["P"], minlength=K)[ks]
    assert np.allclose(p_m, g["psi"] * g["P"] + g["qs"], atol=1e-13, rtol=0)
    rng = np.random.default_rng(0)
    sample = rng.choice(M, 2000, replace=False)
    dq = _per_d(m["Q"][sample][:, None], g["cq"][None, :])
    d2 = dq * dq + (m["P"][sample][:, None] - g["cp"][None, :]) ** 2
    got = d2[np.arange(len(sample)), a[sample]]
    assert np.all(got <= d2.min(axis=1) * (1 + 1e-6) + 1e-12)


def test_invalid_arguments_are_rejected():
    need_gpu()
    import torch
    from paper_2605_21794_gb300 import swpic
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    for args in ((p, p, p, 8, p, p, 0, L, 1), (p, p, p, 8, p, p, 4, -1.0, 1), (p, p, p, -1, p, p, 4, L, 1),
                 (p, p, p, 8, p, p, 4, L, -2)):
        with pytest.raises(swpic.SwpicError):
            swpic.swpic_kmeans_lump(*args, None, p, p, p, p, p, s)
    assert swpic.swpic_kmeans_lump(p, p, p, 0, p, p, 4, L, 3, None, p, p, p, p, p, s) == 0
