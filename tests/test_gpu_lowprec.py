"""Reduced-precision path: FP32 matrix values, basis stored in FP32 or BF16,
FP32 SpMV and orthogonalisation, FP64 sketches and tail (Algorithms 1 and 2).

Two kinds of checks:
* consistency of what the path returns with its own stored basis, against
  the oracle's sketch.  S V_m is an exact fixed-point sketch of the stored
  vectors (40 or more fraction bits below each column's maximum).  S A V_m
  comes from the Arnoldi relation and the FP32 SpMV, so column j deviates from
  S A v_j by the FP32 rounding of one SpMV row sum and one update: at most
  about (w + k + 2) u_32 times the cancellation ratio || |A||v_j| || / ||A v_j||
  (w = widest row, u_32 = 2^-24), checked per column with a factor 4;
* the approximants against the FP64 oracle (O2, same S, m, k and rule): the
  error there is the propagated FP32 / BF16 rounding of the basis.  The FP32
  bound is the 1e-6 target of the workload; the BF16 bound is the observed
  floor (about 4e-3, one BF16 unit roundoff) with a margin.
"""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from workloads.operators import powerlaw_graph_operator
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

BASIS = {"f32": torch.float32, "bf16": torch.bfloat16}


def upload32(skf, A):
    return skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda", dtype=torch.float32)


def arnoldi_lp(skf, A, b, m, k, s, basis, zeta=8, seed=13, identity=False, ldv=None):
    op = upload32(skf, A)
    S = skf.Sketch(skf.IDENTITY if identity else skf.SPARSE_SIGN, A.n, s, zeta, seed)
    info = skf.new_info()
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, k,
                                          basis_dtype=BASIS[basis], info=info, ldv=ldv)
    torch.cuda.synchronize()
    Vn = (V.double() * vs[:, None]).cpu().numpy().T      # stored basis, columns v_j = sigma_j w_j
    return Vn, SV.cpu().numpy().T, SAV.cpu().numpy().T, H.cpu().numpy().T, skf.read_info(info)


def a32(A):
    """The operator with its values rounded to FP32 (what the path multiplies by)."""
    M = csr_to_scipy(A).astype(np.float32).astype(np.float64)
    return M


U32 = 2.0 ** -24


def check_sketches(A, V, SV, SAV, k, s, me):
    S = OSketch("sparse_sign", A.n, s, 8, 13)
    V = V[:, :me]
    assert rel(SV[:, :me], S @ V) < 1e-9
    M = a32(A)
    AV = M @ V
    absAV = abs(M) @ np.abs(V)
    width = int(np.diff(A.rowptr).max())
    SAVo = S @ AV
    for j in range(me):
        err = np.linalg.norm(SAV[:, j] - SAVo[:, j]) / np.linalg.norm(SAVo[:, j])
        bound = 4 * (width + k + 2) * U32 * np.linalg.norm(absAV[:, j]) / np.linalg.norm(AV[:, j])
        assert err <= bound, (j, err, bound)


@pytest.mark.parametrize("basis", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_sketches_are_those_of_the_stored_basis(skf, basis, k):
    A = convdiff_2d(97, (100.0, 50.0))          # N = 9409: ragged last chunk and slice
    b = gaussian_rhs(A.n, 12)
    m, s = 30, 120
    V, SV, SAV, H, info = arnoldi_lp(skf, A, b, m, k, s, basis)
    assert info["status"] == 0 and info["m_eff"] == m
    check_sketches(A, V, SV, SAV, k, s, m)
    # local orthogonality and unit norms of the stored basis, to FP32 accuracy
    G = V.T @ V
    tol = 1e-5 if basis == "f32" else 2e-2
    assert np.abs(np.diag(G) - 1.0).max() < tol
    for j in range(m):
        for i in range(max(0, j - k + 1), j):
            assert abs(G[i, j]) < tol, (i, j, G[i, j])


def test_sketches_wide_rows_graph_operator(skf):
    """Rows wider than eight entries (several passes of the SpMV row loop)."""
    A = powerlaw_graph_operator(6000, seed=11)
    widths = np.diff(A.rowptr)
    assert widths.max() > 16
    b = gaussian_rhs(A.n, 12)
    m, s = 20, 80
    for basis in ("f32", "bf16"):
        V, SV, SAV, H, info = arnoldi_lp(skf, A, b, m, 3, s, basis)
        assert info["status"] == 0 and info["m_eff"] == m
        check_sketches(A, V, SV, SAV, 3, s, m)


@pytest.mark.parametrize("m", [1, 2, 5])
def test_short_bases(skf, m):
    """m = 1 (the only column is the last: S y_0 scattered directly) and short
    bases where the relation and the direct column meet."""
    A = convdiff_2d(40)
    b = gaussian_rhs(A.n, 12)
    V, SV, SAV, H, info = arnoldi_lp(skf, A, b, m, 2, 4 * m + 8, "f32")
    assert info["m_eff"] == m
    check_sketches(A, V, SV, SAV, 2, 4 * m + 8, m)


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_identity_sketch(skf, basis):
    A = convdiff_2d(20)
    b = gaussian_rhs(A.n, 3)
    V, SV, SAV, H, info = arnoldi_lp(skf, A, b, 12, 2, A.n, basis, identity=True)
    assert info["m_eff"] == 12
    assert rel(SV, V) < 1e-15
    assert rel(SAV, a32(A) @ V) < 2e-6


def solve_lp(skf, A, b, func, m, k, s, c, method, basis, tol=1e-12):
    op = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    f = skf.make_func(func, c)
    p = skf.make_params(m, k, basis_dtype=BASIS[basis], tol=tol)
    info = skf.new_info()
    x = skf.solve(method, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    return x.cpu().numpy(), skf.read_info(info)


# FP32: the 1e-6 target of the reduced-precision workload; BF16: the floor of
# about one BF16 unit roundoff (3.9e-3) with a margin
BOUND = {"f32": 1e-6, "bf16": 3e-2}


@pytest.mark.parametrize("basis", ["f32", "bf16"])
@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_config1_against_fp64_oracle(skf, basis, method):
    """2D convection-diffusion N = 1e4, m = 40, k = 2, s = 160, z^{-1/2}."""
    A = convdiff_2d(100, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 40, 2, 160
    x, info = solve_lp(skf, A, b, "invsqrt", m, k, s, c, skf.SGMRES if method == "sgmres" else skf.SFOM, basis)
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    assert info["status"] == 0 and info["m_eff"] == m
    err = rel(x, xo)
    print(f"{basis} {method}: rel err vs FP64 oracle {err:.3e}")
    assert err <= BOUND[basis]


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_3d_log1p_against_fp64_oracle(skf, basis):
    A = convdiff_3d(24, (50.0, 50.0, 50.0))     # N = 13824
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("log1p_over_z", 0.0, float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 50, 2, 200
    x, info = solve_lp(skf, A, b, "log1p_over_z", m, k, s, c, skf.SGMRES, basis)
    xo, _ = osk.solve(csr_to_scipy(A), b, "log1p_over_z", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres", tol=1e-12)
    assert info["status"] == 0
    err = rel(x, xo)
    print(f"{basis} 3d log1p sgmres: rel err vs FP64 oracle {err:.3e}")
    assert err <= BOUND[basis]


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_zero_rhs(skf, basis):
    A = convdiff_2d(16)
    op = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 64, 8, 13)
    f = skf.make_func("invsqrt", 1.0)
    p = skf.make_params(8, 2, basis_dtype=BASIS[basis])
    info = skf.new_info()
    x = skf.solve(skf.SGMRES, op.csr, S, torch.zeros(A.n, dtype=torch.float64, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    st = skf.read_info(info)
    assert st["status_name"] == "SKF_ERR_ZERO_RHS"
    assert float(x.abs().max()) == 0.0


def test_invariant_subspace_breakdown_fp32(skf):
    """A = diag with 5 distinct values: the Krylov space is invariant after 5
    steps, which the FP32 test (||w|| <= 2^-17 ||A v||) detects."""
    from workloads.operators import CSR
    N = 640
    d = np.repeat(np.array([1.0, 2.0, 3.0, 5.0, 8.0]), N // 5)
    A = CSR(N, np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32), d)
    b = gaussian_rhs(N, 12)
    V, SV, SAV, H, info = arnoldi_lp(skf, A, b, 12, 12, 64, "f32")
    assert info["breakdown"] == 1 and info["m_eff"] == 5
    # the columns before the breakdown, including S A v_4 from the relation
    check_sketches(A, V, SV, SAV, 12, 64, 5)


def test_mixed_dtypes_rejected(skf):
    A = convdiff_2d(16)
    op64 = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    op32 = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 64, 8, 13)
    b = torch.as_tensor(gaussian_rhs(A.n, 12), device="cuda")
    with pytest.raises(skf.SkfError):
        skf.arnoldi_trunc(op64.csr, S, b, 8, 2, basis_dtype=torch.float32)
    with pytest.raises(skf.SkfError):
        skf.arnoldi_trunc(op32.csr, S, b, 8, 2, basis_dtype=torch.float64)


@pytest.mark.parametrize("basis", ["f32", "bf16"])
@pytest.mark.parametrize("n,ldv", [(90, None), (1010, 1020160)])
def test_many_chunks_per_cta(skf, basis, n, ldv):
    """Five or more 1024-row chunks per CTA (the pipelined SpMV carries column
    indices and slice metadata from chunk to chunk): 3D n = 90 (N = 729000)
    and 2D n = 1010 (N = 1020100, ragged last chunk) with a padded leading
    dimension.  Basis and sketches against the oracle."""
    from oracle.arnoldi import arnoldi_trunc as o_arnoldi
    A = convdiff_3d(n, (50.0, 50.0, 50.0)) if n == 90 else convdiff_2d(n, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    m, k, s = 8, 2, 48
    V, SV, SAV, H, info = arnoldi_lp(skf, A, b, m, k, s, basis, ldv=ldv)
    assert info["status"] == 0 and info["m_eff"] == m
    check_sketches(A, V, SV, SAV, k, s, m)
    if basis == "f32":
        ar = o_arnoldi(a32(A), b, m, k, OSketch("sparse_sign", A.n, s, 8, 13))
        for j in range(m):   # FP32 recurrence against the FP64 one: a few hundred u_32 after 8 steps
            assert rel(V[:, j], ar["V"][:, j]) < 1e-4, j


@pytest.mark.parametrize("zeta", [4, 8, 12])
def test_sketch_sparsity_variants(skf, zeta):
    """zeta = 8 takes the compact-pattern split bins; 4 and 12 the general ones."""
    A = convdiff_2d(60)
    b = gaussian_rhs(A.n, 12)
    m, s = 12, 96
    op = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, zeta, 13)
    info = skf.new_info()
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, 2,
                                          basis_dtype=torch.float32, info=info)
    torch.cuda.synchronize()
    Vn = (V.double() * vs[:, None]).cpu().numpy().T
    So = OSketch("sparse_sign", A.n, s, zeta, 13)
    assert rel(SV.cpu().numpy().T, So @ Vn) < 1e-9
    assert rel(SAV.cpu().numpy().T, So @ (a32(A) @ Vn)) < 1e-5


def test_graph_fixed_rule_128_nodes(skf):
    """The quadrature-batched form of the graph workload: a directed power-law
    graph operator (A = D_s + 0.1 I - W^T), FP32 values and basis, k = 3, and
    sGMRES with a fixed 128-node Gauss-Jacobi rule whose nodes are solved in
    one batch.  On this operator (hub rows make it strongly non-normal and
    badly scaled) the truncated basis loses independence quickly and the FP32
    rounding of each new basis vector is amplified by its conditioning, so the
    FP32 result differs from the FP64 approximant by far more than on the
    convection-diffusion operators.  The check is therefore against the exact
    f(A)b (dense, N = 2000; the 128-node rule's own error is far below the
    Krylov errors compared): the FP32 approximant may be at most twice as far
    from it as the FP64 one."""
    from oracle.quadrature import rule
    A = powerlaw_graph_operator(2000, seed=11)
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", 0.1, float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 30, 3, 120
    t, w = rule("invsqrt", 128, c)
    op = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    f = skf.make_func("invsqrt", c, nodes=t, weights=w)
    p = skf.make_params(m, k, basis_dtype=torch.float32)
    info = skf.new_info()
    x = skf.solve(skf.SGMRES, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    st = skf.read_info(info)
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres", ell=128)
    assert st["status"] == 0 and st["m_eff"] == m
    from oracle.exact import fAb_dense
    xq = fAb_dense(csr_to_scipy(A).toarray(), b, "invsqrt")   # exact f(A) b (dense Schur-based)
    x32 = x.cpu().numpy()
    e32, e64, d = rel(x32, xq), rel(xo, xq), rel(x32, xo)
    print(f"graph 128-node sgmres: err f32 {e32:.3e}, err f64 {e64:.3e}, f32 vs f64 {d:.3e}, "
          f"rdiag_ratio {st['rdiag_ratio']:.3e}")
    assert e32 <= 2.0 * e64 + 1e-6


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_f32_relation_form_equals_full_form(skf, k, method):
    """FP32 basis: its S A v_j (j < m - 1) are formed from the sketched Arnoldi
    relation with the coefficients the update applied, so the relation-form
    tail (QR of [S V_m, S A v_m], M = [R_11 H, r] R_11^{-1}) and the full form
    (QR of [S V_m, S A V_m]) factor the same sketched relation and agree to
    FP64 rounding times cond(R); both stay within max(1e-6, 2^-24 cond(R)) of
    the FP64 oracle."""
    A = convdiff_2d(100, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    m = 16 if k == 1 else 40
    s = 4 * m
    meth = skf.SGMRES if method == "sgmres" else skf.SFOM
    x_rel, i_rel = solve_lp(skf, A, b, "invsqrt", m, k, s, c, meth, "f32")
    with skf.tail_form(skf.TAIL_FULL):
        x_full, i_full = solve_lp(skf, A, b, "invsqrt", m, k, s, c, meth, "f32")
    xo, oi = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    assert i_rel["status"] == 0 and i_full["status"] == 0
    assert i_rel["ell"] == i_full["ell"]
    d = rel(x_rel, x_full)
    print(f"f32 k={k} {method}: relation vs full {d:.3e}, cond_est {i_rel['cond_est']:.3e}, "
          f"vs oracle {rel(x_rel, xo):.3e}")
    assert d <= max(1e-10, 1e-14 * i_rel["cond_est"])
    # against the FP64 oracle: the FP32 basis moves the approximant by about
    # 2^-24 cond(R) (k = 1 loses basis independence fastest: cond(R) ~ 9e2 here)
    bound = max(BOUND["f32"], 2.0 ** -24 * i_rel["cond_est"])
    assert rel(x_rel, xo) <= bound and rel(x_full, xo) <= bound


@pytest.mark.parametrize("kind", ["srht", "srdct"])
def test_f32_basis_dense_sketches(skf, kind):
    """An FP32 basis with the SRHT or the paper's SRDCT (Sec. 5.1): S v_j is the
    sketch of the stored basis (computed in FP64 from the widened FP32 values,
    the SRHT exactly), S A v_j the sketch of the FP32 SpMV result (within the
    FP32 rounding of A v_j), and both solves stay within
    max(1e-6, 2^-24 cond(R)) of the FP64 oracle with the same sketch."""
    A = convdiff_2d(100, (100.0, 50.0))          # N = 1e4 = 2^4 5^4: the SRDCT takes its FFT form
    b = gaussian_rhs(A.n, 12)
    m, k, s = 40, 2, 160
    op = upload32(skf, A)
    kinds = {"srht": skf.SRHT, "srdct": skf.SRDCT}
    S = skf.Sketch(kinds[kind], A.n, s, 0, 13)
    OS = OSketch(kind, A.n, s, seed=13)
    bt = torch.as_tensor(b, device="cuda")
    info = skf.new_info()
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, bt, m, k, basis_dtype=torch.float32, info=info)
    torch.cuda.synchronize()
    assert skf.read_info(info)["status"] == 0
    Vn = (V.double() * vs[:, None]).cpu().numpy().T
    SVg, SAVg = SV.cpu().numpy().T, SAV.cpu().numpy().T
    assert rel(SVg, OS @ Vn) < 1e-12
    M = a32(A)
    AV = M @ Vn
    width = int(np.diff(A.rowptr).max())
    for j in range(m):
        err = np.linalg.norm(SAVg[:, j] - OS @ AV[:, j]) / np.linalg.norm(OS @ AV[:, j])
        bound = 4 * (width + k + 2) * U32 * np.linalg.norm(abs(M) @ np.abs(Vn[:, j])) / np.linalg.norm(AV[:, j])
        assert err <= bound, (j, err, bound)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    for meth, om in ((skf.SGMRES, "sgmres"), (skf.SFOM, "sfom_quad")):
        inf = skf.new_info()
        x = skf.solve(meth, op.csr, S, bt, f, skf.make_params(m, k, basis_dtype=torch.float32, tol=1e-12), info=inf)
        xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OS, c, method=om, tol=1e-12)
        torch.cuda.synchronize()
        st = skf.read_info(inf)
        err = rel(x.cpu().numpy(), xo)
        print(f"f32 {kind} {om}: rel err vs FP64 oracle {err:.3e}, cond_est {st['cond_est']:.3e}")
        assert st["status"] == 0
        assert err <= max(BOUND["f32"], U32 * st["cond_est"])


def test_bf16_basis_dense_sketch_not_supported(skf):
    A = convdiff_2d(20)
    op = upload32(skf, A)
    S = skf.Sketch(skf.SRHT, A.n, 40, 0, 13)
    with pytest.raises(skf.SkfError, match="NOT_SUPPORTED"):
        skf.arnoldi_trunc(op.csr, S, torch.as_tensor(gaussian_rhs(A.n, 1), device="cuda"), 8, 2,
                          basis_dtype=torch.bfloat16)


@pytest.mark.parametrize("basis", ["f64", "f32"])
def test_returned_h_is_the_relation_of_the_stored_basis(skf, basis):
    """H as skf_arnoldi_trunc returns it holds the Arnoldi relation (eq. (2.1))
    of the stored, normalised basis: S A v_j = S V_{j+2} H(:, j) for j < m - 1
    to FP64 rounding (the FP32 path forms those S A v_j from that very
    relation), and A v_j = V H(:, j) to the basis precision (FP64: rounding of
    the recurrence; FP32: the FP32 SpMV and update)."""
    A = convdiff_2d(60, (80.0, 20.0))
    b = gaussian_rhs(A.n, 9)
    m, k, s = 30, 2, 120
    if basis == "f32":
        op = upload32(skf, A)
        M = a32(A)
    else:
        op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
        M = csr_to_scipy(A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, k,
                                          basis_dtype=torch.float32 if basis == "f32" else torch.float64)
    torch.cuda.synchronize()
    Vn = (V.double() * vs[:, None]).cpu().numpy().T
    SVn, SAVn, Hn = SV.cpu().numpy().T, SAV.cpu().numpy().T, H.cpu().numpy().T   # H: (m + 1) x m
    sk = SVn[:, :m] @ Hn[:m, : m - 1]
    d_sk = np.linalg.norm(sk - SAVn[:, : m - 1]) / np.linalg.norm(SAVn[:, : m - 1])
    AV = M @ Vn[:, : m - 1]
    R = AV - Vn[:, :m] @ Hn[:m, : m - 1]
    d_rel = np.linalg.norm(R) / np.linalg.norm(AV)
    print(f"{basis}: sketched relation {d_sk:.2e}, relation {d_rel:.2e}")
    assert d_sk <= 1e-12
    if basis == "f64":
        assert d_rel <= 1e-13
    else:
        # per column: the FP32 SpMV and update roundings, as in check_sketches
        width = int(np.diff(A.rowptr).max())
        absAV = abs(M) @ np.abs(Vn[:, : m - 1])
        for j in range(m - 1):
            bound = 4 * (width + k + 2) * U32 * np.linalg.norm(absAV[:, j]) / np.linalg.norm(AV[:, j])
            assert np.linalg.norm(R[:, j]) / np.linalg.norm(AV[:, j]) <= bound, j


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_f32_persistent_and_two_kernel_forms(skf, method):
    """An FP32 basis in the persistent Arnoldi form (FP32 SpMV and update in one
    cooperative launch, the window on chip) and in the two-kernel form: the
    sketches are those of each stored basis, and both solves stay within
    max(1e-6, 2^-24 cond(R)) of the FP64 oracle."""
    A = convdiff_2d(100, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 40, 2, 160
    op = upload32(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    f = skf.make_func("invsqrt", c)
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    xs = {}
    for form in (skf.ARNOLDI_PERSISTENT, skf.ARNOLDI_TWO_KERNEL):
        with skf.arnoldi_mode(form):
            V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, k,
                                                  basis_dtype=torch.float32)
            info = skf.new_info()
            x = skf.solve(skf.SGMRES if method == "sgmres" else skf.SFOM, op.csr, S,
                          torch.as_tensor(b, device="cuda"), f,
                          skf.make_params(m, k, basis_dtype=torch.float32, tol=1e-12), info=info)
            torch.cuda.synchronize()
        Vn = (V.double() * vs[:, None]).cpu().numpy().T
        check_sketches(A, Vn, SV.cpu().numpy().T, SAV.cpu().numpy().T, k, s, m)
        st = skf.read_info(info)
        err = rel(x.cpu().numpy(), xo)
        print(f"f32 form {form} {method}: rel err vs FP64 oracle {err:.3e}, cond_est {st['cond_est']:.3e}")
        assert st["status"] == 0
        assert err <= max(BOUND["f32"], U32 * st["cond_est"])
        xs[form] = x.cpu().numpy()
    assert rel(xs[skf.ARNOLDI_PERSISTENT], xs[skf.ARNOLDI_TWO_KERNEL]) <= 2e-6
