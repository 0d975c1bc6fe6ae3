"""Parity at the full sizes of the bench's extra lines, on outputs the oracle
can compute one by one (the operator is separable over transducers for A,
Alg. 1, and over voxels for A^T, Alg. 5):
  * c3 (256^3 voxels @ 0.08 mm, the first 128 planar positions, tcgen05 BF16
    split convolution, as the precision-split line): two whole rows of s over
    all 16.7M voxels, bar 1e-3 (the reduced-precision bound; the geometric
    part alone is FP32), and A^T at 256 seeded voxels;
  * c5 (512^3 voxels @ 0.05 mm, the first 16 cylindrical positions, closed
    form, as the full-scale line): one whole row of s over all 134M voxels and
    A^T at 128 seeded voxels, bar 1e-5, and the dot-product identity over the
    whole output;
  * Exp-1 fine (98,415 voxels x 215 cylindrical elements) with the paper's
    1000 x 1000 lookup tables, as the N4 line: four whole rows of s and A^T at
    256 voxels, bar 1e-5.
The system-kernel taps come from the oracle on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

FP32_TOL = 1e-5
TC_TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29253_gb300 import api as A

    return A


def _rows(orc, w, taps, ks):
    x64 = w.x.astype(np.float64)
    out = []
    for k in ks:
        s_ref, dropped = orc.forward(w.with_tx(w.tx[k:k + 1]), taps, x64)
        assert dropped == 0
        out.append(s_ref[0])
    return np.stack(out)


def _adjoint_sample(orc, plan, w, taps, n_vox, seed, tol):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal((w.K, w.L)).astype(np.float32)
    z = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    idx = np.sort(rng.choice(w.N, size=n_vox, replace=False)).astype(np.int64)
    z_ref, dropped = orc.adjoint(w, taps, y.astype(np.float64), vox_idx=idx)
    assert dropped == 0
    e = rel(z[idx], z_ref)
    print(f"A^T at {n_vox} voxels: rel L2 {e:.3e}")
    assert e <= tol, e


def test_c3_precision_split_full_size(api, oracle_mod):
    w = W.c3(with_x=False, rotations=1)
    w = w.with_tx(w.tx[:128])
    w = w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True)
    s = plan.forward(torch.from_numpy(w.x).cuda()).cpu().numpy()
    ks = np.array([5, 77])
    e = rel(s[ks], _rows(oracle_mod, w, taps, ks))
    print(f"c3 rows {ks.tolist()}: rel L2 {e:.3e}")
    assert e <= TC_TOL, e
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0
    _adjoint_sample(oracle_mod, plan, w, taps, 256, 5, TC_TOL)


def test_c5_full_scale_subset(api, oracle_mod):
    w = W.c5(with_x=False, n_angles=128)
    w = w.with_tx(w.tx[:16])
    w = w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps)
    x = torch.from_numpy(w.x).cuda()
    s = plan.forward(x)
    ks = np.array([9])
    e = rel(s.cpu().numpy()[ks], _rows(oracle_mod, w, taps, ks))
    print(f"c5 row {ks.tolist()}: rel L2 {e:.3e}")
    assert e <= FP32_TOL, e
    _adjoint_sample(oracle_mod, plan, w, taps, 128, 6, FP32_TOL)
    g = torch.Generator(device="cuda").manual_seed(4)
    y = torch.randn(w.K, w.L, device="cuda", generator=g)
    lhs = float((s.double() * y.double()).sum())
    rhs = float((x.double() * plan.adjoint(y).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_exp1_lookup_tables_full_size(api, oracle_mod):
    w = W.exp1("fine", method=W.METHOD_LUT)
    assert (w.q1, w.q2) == (1000, 1000)
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps)
    s = plan.forward(torch.from_numpy(w.x).cuda()).cpu().numpy()
    ks = np.array([0, 50, 107, 214])
    e = rel(s[ks], _rows(oracle_mod, w, taps, ks))
    print(f"Exp-1 LUT rows {ks.tolist()}: rel L2 {e:.3e}")
    assert e <= FP32_TOL, e
    _adjoint_sample(oracle_mod, plan, w, taps, 256, 7, FP32_TOL)
