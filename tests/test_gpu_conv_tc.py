"""GPU parity of the tensor-core (tcgen05) temporal convolution, plans created
with PAT_FLAG_CONV_TC, against the FP64 oracle, through the C ABI.

The convolution runs with BF16 operands split in two (x = hi + lo) and the
products hi*hi + hi*lo + lo*hi accumulated in FP32, so each product keeps
about 16 significant bits.  Bound: rel L2 <= 1e-4 on every stage and on the
whole A and A^T (the target for the reduced-precision convolution is 1e-3; a
single BF16 pass gives about 1e-2 on these kernels because Sum h-bar = 0
makes the outputs small against the terms).  Sizes span several 128-sample
output tiles, a ragged last tile, a ragged transducer tile (K not a multiple
of 64) and more than one transducer tile.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

TC_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29253_gb300 import api as A

    return A


def _stages(api, orc, w, seed):
    taps = orc.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True, allow_clip=True)  # the stages alone: any time window
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((w.K, w.UL)).astype(np.float32)
    s = plan.conv_forward(torch.from_numpy(f).cuda()).cpu().numpy()
    s_ref = orc.conv_forward(w, taps, f.astype(np.float64))
    y = rng.standard_normal((w.K, w.L)).astype(np.float32)
    v = plan.conv_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    v_ref = orc.conv_adjoint(w, taps, y.astype(np.float64))
    assert plan.info["tc_error"] == 0 and api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0
    return rel(s, s_ref), rel(v, v_ref)


@pytest.mark.parametrize("L,n_angles,n_el", [(1024, 2, 3), (300, 10, 8), (129, 3, 43), (1024, 8, 40), (1024, 10, 64)])
def test_conv_stages_tensor_cores(api, oracle_mod, L, n_angles, n_el):
    """f -> s and s -> v alone: L = 1024 (8 tiles), 300 (ragged), 129 (one
    sample in the last tile); K = 6, 80 (two transducer tiles), 129, and 320
    and 640, where each CTA of the forward kernel runs its ring of stage
    buffers several times over (40 tiles with the stages split in three; 80
    tiles, every stage in one CTA)."""
    w = W.small_cylinder(n_vox=4, n_angles=n_angles, n_el=n_el, L=L)
    es, ev = _stages(api, oracle_mod, w, seed=L)
    assert es <= TC_TOL, es
    assert ev <= TC_TOL, ev


def test_conv_stages_planar_taps(api, oracle_mod):
    """The planar c1 system's kernel (another tap window)."""
    es, ev = _stages(api, oracle_mod, W.c1(), seed=3)
    assert es <= TC_TOL and ev <= TC_TOL, (es, ev)


@pytest.mark.parametrize("mk", ["plane", "cylinder"])
def test_operator_tensor_cores(api, oracle_mod, mk):
    w = W.c1() if mk == "plane" else W.small_cylinder(n_vox=10, n_angles=4, n_el=3)
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True)
    x32 = w.x.astype(np.float32)
    s = plan.forward(torch.from_numpy(x32).cuda()).cpu().numpy()
    s_ref, _ = oracle_mod.forward(w, taps, x32.astype(np.float64))
    assert rel(s, s_ref) <= TC_TOL, rel(s, s_ref)
    y = np.random.default_rng(8).standard_normal(s.shape).astype(np.float32)
    z = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref, _ = oracle_mod.adjoint(w, taps, y.astype(np.float64))
    assert rel(z, z_ref) <= TC_TOL, rel(z, z_ref)
    # the FP32 / FP64-accumulation convolution of the plain plan agrees too
    plain = api.Plan(w, taps=taps)
    s2 = plain.forward(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert rel(s, s2) <= TC_TOL
    assert plan.info["tc_error"] == 0 and api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0


def test_adjoint_tensor_cores_physical_scale(api, oracle_mod):
    """A^T of the operator's own output, s = A x of order 1e-16 for x of order
    1 (the system kernel in SI units is of order 1e-20): v = h-bar^- * s is then
    near 1e-36, and the products of the BF16 split, about 2^-8 of v, would fall
    below FP32's smallest normal (1.2e-38) in the tensor cores; the operand
    tables carry a power-of-two scale that keeps them of the signal's size.
    Checked on the stage (v) and on the whole A^T (z)."""
    w = W.small_cylinder(n_vox=10, n_angles=4, n_el=3)
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True)
    s_ref, _ = oracle_mod.forward(w, taps, w.x.astype(np.float64))
    s32 = s_ref.astype(np.float32)
    assert 1e-18 < float(np.abs(s32).max()) < 1e-13
    v = plan.conv_adjoint(torch.from_numpy(s32).cuda()).cpu().numpy()
    v_ref = oracle_mod.conv_adjoint(w, taps, s32.astype(np.float64))
    assert float(np.abs(v_ref).max()) < 1e-33  # the regime in question
    assert rel(v, v_ref) <= TC_TOL, rel(v, v_ref)
    z = plan.adjoint(torch.from_numpy(s32).cuda()).cpu().numpy()
    z_ref, _ = oracle_mod.adjoint(w, taps, s32.astype(np.float64))
    assert rel(z, z_ref) <= TC_TOL, rel(z, z_ref)
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0


def test_dot_product_tensor_cores(api, oracle_mod):
    w = W.small_cylinder(n_vox=8, n_angles=4, n_el=3)
    plan = api.Plan(w, taps=oracle_mod.taps_for(w), conv_tc=True)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(w.N, device="cuda", generator=g)
    y = torch.randn(w.K, w.L, device="cuda", generator=g)
    lhs = float((plan.forward(x).double() * y.double()).sum())
    rhs = float((x.double() * plan.adjoint(y.contiguous()).double()).sum())
    assert abs(lhs - rhs) <= TC_TOL * abs(lhs)


def test_recon_with_tensor_core_plan(api, oracle_mod):
    w = W.c1().with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True)
    xt = torch.from_numpy(W.uniform_phantom(512, 7)).cuda()
    s = plan.forward(xt)
    x0 = torch.zeros(512, device="cuda")
    r0 = float((plan.forward(x0) - s).norm())
    x30 = plan.recon(s, x0, iters=30, lambda_R=0.0)
    r30 = float((plan.forward(x30) - s).norm())
    assert float(x30.min()) >= 0.0 and r30 < 0.5 * r0


# ---------------------------------------------------------------------------
# Split-plane forward (the kernel pat_forward uses on tensor-core plans): f as
# BF16 hi and lo planes, 128 x 256 tiles brought in by tensor-map copies,
# persistent CTAs with two TMEM accumulators.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,n_angles,n_el", [(1024, 2, 3), (300, 10, 8), (129, 3, 43), (1024, 8, 40),
                                             (2048, 20, 128)])
def test_conv_forward_split_planes(api, oracle_mod, L, n_angles, n_el):
    """L = 1024, 300 (ragged last tile, a row length that is not a multiple
    of 8 fine bins: 3300), 129; K = 6, 80, 129 (inside one 256-row tile),
    320 (two tiles, the second ragged) and 2560 with L 2048 (10 x 16 = 160
    tiles: more than one per CTA, both accumulators and both ring slots
    cycling)."""
    w = W.small_cylinder(n_vox=4, n_angles=n_angles, n_el=n_el, L=L)
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True, allow_clip=True)
    rng = np.random.default_rng(L + n_el)
    f = rng.standard_normal((w.K, w.UL)).astype(np.float32)
    ft = torch.from_numpy(f).cuda()
    planes = plan.conv_split(ft)
    s = plan.conv_forward_split(planes).cpu().numpy()
    s_ref = oracle_mod.conv_forward(w, taps, f.astype(np.float64))
    e = rel(s, s_ref)
    print(f"K {w.K} L {L}: split-plane forward rel L2 {e:.3e}")
    assert e <= TC_TOL, e
    # the same split products as the FP32-input kernel: agreement to FP32 accumulation order
    s_fp32in = plan.conv_forward(ft).cpu().numpy()
    assert rel(s, s_fp32in) <= 1e-5, rel(s, s_fp32in)
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0


def test_split_planes_layout(api, oracle_mod):
    """hi = bf16(f), lo = bf16(f - hi), rows of ld = U L rounded up to 8, zero padding."""
    w = W.small_cylinder(n_vox=4, n_angles=3, n_el=4, L=300)
    plan = api.Plan(w, taps=oracle_mod.taps_for(w), conv_tc=True, allow_clip=True)
    f = torch.randn(w.K, w.UL, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    planes = plan.conv_split(f)
    ld = -(-w.UL // 8) * 8
    assert planes.numel() * 2 >= 2 * w.K * ld * 2
    p = planes[:2 * w.K * ld].view(2, w.K, ld)
    hi = p[0].view(torch.bfloat16).float()
    lo = p[1].view(torch.bfloat16).float()
    assert torch.equal(hi[:, :w.UL], f.to(torch.bfloat16).float())
    assert torch.equal(lo[:, :w.UL], (f - hi[:, :w.UL]).to(torch.bfloat16).float())
    assert float(p[:, :, w.UL:].abs().max()) == 0.0


def test_split_plane_give_up_path(api, oracle_mod):
    """The bounded waits of the tensor-core kernels, made to run out without a
    fault or an endless wait: with the release of the first accumulator
    withheld, the MMA warp gives up at the third tile after about two seconds;
    the kernel stops, frees its TMEM and reports through tc_error.  The plan
    stays usable: after clearing the error, the next call matches the FP64
    convolution with tc_error 0."""
    w = W.small_cylinder(n_vox=4, n_angles=2, n_el=3, L=1024)  # 8 output tiles, one CTA
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps, conv_tc=True, allow_clip=True)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((w.K, w.UL)).astype(np.float32)
    planes = plan.conv_split(torch.from_numpy(f).cuda())
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0
    plan.conv_forward_split_withheld(planes)
    torch.cuda.synchronize()
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] != 0
    plan.clear_tc_error()
    torch.cuda.synchronize()
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0
    s = plan.conv_forward_split(planes).cpu().numpy()
    s_ref = oracle_mod.conv_forward(w, taps, f.astype(np.float64))
    assert rel(s, s_ref) <= TC_TOL, rel(s, s_ref)
    assert api._lib.pat_plan_get_info(plan.handle)["tc_error"] == 0


def test_give_up_test_needs_three_tiles(api, oracle_mod):
    """pat_conv_forward_split_withheld refuses a plan whose single CTA would not
    reach the withheld accumulator (fewer than 3 output tiles)."""
    w = W.small_cylinder(n_vox=4, n_angles=2, n_el=3, L=256)  # 2 output tiles
    plan = api.Plan(w, taps=oracle_mod.taps_for(w), conv_tc=True, allow_clip=True)
    planes = plan.conv_split(torch.zeros(w.K, w.UL, device="cuda"))
    with pytest.raises(Exception, match="3 output tiles"):
        plan.conv_forward_split_withheld(planes)
