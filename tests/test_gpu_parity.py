"""GPU parity: every step of the hot path, through the C ABI, against the CPU oracle.

Bars: sampled indices and gathered fibers bit-exact; updated factors within 1e-4 relative
Frobenius for FP32/BF16 tensors (FP32 contraction) and 1e-10 for FP64 tensors; whole runs reach
the oracle's final fit within 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import cp, mixing, streams
from synth import make_problem, to_oracle_array
from fp32_floor import fp32_product_floor, fp32_trace_floor

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def cb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding
    return binding


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture
def engine(cb):
    """Sets the process-wide mixing engine for one test and restores the previous one afterwards."""
    prev = cb.cpr_set_mix_engine(cb.MIX_AUTO)
    yield cb.cpr_set_mix_engine
    cb.cpr_set_mix_engine(prev)


def assert_elementwise(got, ref, eps, depth):
    """Every entry of a mixed tensor within eps * (|ref_i| + depth * rms(ref)) of the oracle's.

    Mixing is a chain of orthonormal mode products, so the rounding a pass commits in one fiber is
    spread by the later passes over the whole tensor at the scale of the entries' root mean square;
    depth counts the rounding steps an entry accumulates (passes x transform depth).  A wrong entry,
    or a wrong block of entries, is off by about rms(ref) and fails this bound at any size, where a
    relative Frobenius bound over the whole tensor could absorb it."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    rms = np.linalg.norm(ref) / np.sqrt(ref.size)
    bound = eps * (np.abs(ref) + depth * rms)
    excess = np.abs(got - ref) / bound
    worst = np.unravel_index(int(np.argmax(excess)), ref.shape)
    assert excess[worst] <= 1.0, ("entry", worst, float(got[worst]), float(ref[worst]), float(excess[worst]))


def rand_tensor(dims, dtype, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(int(np.prod(dims)), generator=g, dtype=torch.float64).to(dtype).to(DEV)


# ------------------------------------------------------------------------------------------------
# a1: sampler (bit-exact)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims,n,S,t,b", [
    ((400, 400, 400), 0, 230, 0, 0), ((400, 400, 400), 2, 230, 7, 0), ((100, 100, 100, 100), 1, 450, 3, 2),
    ((7, 1, 13, 5, 3, 2), 3, 1000, 1, 1), ((64, 512, 300), 1, 1109, 199, 63), ((50, 50, 50), 1, 80, 49, 0),
    ((1500, 1500, 1500), 1, 2000, 11, 0), ((3, 4, 5, 6, 7, 8, 9, 10), 7, 4096, 2, 5), ((9, 9), 0, 0, 0, 0)])
def test_sampler_bit_exact(cb, dims, n, S, t, b):
    seed = 2001
    idx, off = cb.cpr_sample_indices(dims, n, S, seed, b, t)
    torch.cuda.synchronize()
    ref = streams.ls_sample_indices(seed, b, t, n, S, dims)
    np.testing.assert_array_equal(idx.cpu().numpy().astype(np.int64), ref)
    if S:
        ref_off = np.ravel_multi_index(tuple(ref[:, m] for m in range(len(dims))), dims, order="F")
        np.testing.assert_array_equal(off.cpu().numpy(), ref_off)


# ------------------------------------------------------------------------------------------------
# a2: fiber gather (bit-exact)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
@pytest.mark.parametrize("dims", [(37, 29, 41), (1, 30, 20), (11, 7, 5, 9, 3), (64, 40, 24), (400, 13, 11)])
def test_gather_bit_exact(cb, dtype, dims):
    # first-mode fibers of 64 or 400 entries take the 16-byte vector path (whole-warp fibers)
    X = rand_tensor(dims, dtype, 1)
    T = to_oracle_array(X, dims)
    for n in range(len(dims)):
        idx, off = cb.cpr_sample_indices(dims, n, 77, 9, 0, n)
        Xs = cb.cpr_gather_fibers(X, dims, n, off)
        torch.cuda.synchronize()
        ref = cp.gather_fibers(T, idx.cpu().numpy().astype(np.int64), n)
        got = Xs.float().cpu().double().numpy() if dtype == torch.bfloat16 else Xs.cpu().double().numpy()
        np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------------------------------------
# a1-a6: one mode update of Alg. 3
# ------------------------------------------------------------------------------------------------
UPDATE_CASES = [
    # dims, R, S, dtype, tol
    ((37, 29, 41), 4, 60, torch.float32, 1e-4),
    ((70, 130, 65), 7, 100, torch.bfloat16, 1e-4),
    ((50, 50, 50), 5, 80, torch.float64, 1e-10),
    ((9, 8, 7, 6, 5, 4), 3, 40, torch.float32, 1e-4),
    ((80, 70, 90), 64, 128, torch.float32, 1e-4),      # R = CPR_MAX_RANK
    ((300, 280, 290), 8, 8, torch.float32, 1e-4),      # S = R (no repeated sample rows here)
    ((1, 30, 20), 1, 5, torch.float32, 1e-4),          # I_1 = 1, R = 1
    ((400, 400, 400), 10, 230, torch.float32, 1e-4),   # full size of the 400^3 workload
]


@pytest.mark.parametrize("dims,R,S,dtype,tol", UPDATE_CASES)
def test_sampled_update_matches_oracle(cb, dims, R, S, dtype, tol):
    prob = make_problem(dims, min(R, min(dims)), C=0.5, eta=0.01, seed=3, dtype=dtype, device=DEV)
    T = to_oracle_array(prob.X, dims)
    rng = np.random.default_rng(4)
    if dtype == torch.float64:
        f0 = [rng.random((d, R)) for d in dims]
    else:
        f0 = [rng.random((d, R)).astype(np.float32).astype(np.float64) for d in dims]
    for n in range(len(dims)):
        facs = [torch.tensor(f, device=DEV) for f in f0]
        lam = torch.empty(R, dtype=torch.float64, device=DEV)
        st = cb.cpr_sampled_update(prob.X, dims, lam, facs, n, S, seed=77, b=1, t=5 + n)
        assert st == cb.OK
        idx = streams.ls_sample_indices(77, 1, 5 + n, n, S, dims)
        A_ref, lam_ref = cp.cprand_update(T, f0, n, idx)
        assert rel(facs[n].cpu().numpy(), A_ref) < tol, n
        assert rel(lam.cpu().numpy(), lam_ref) < tol, n


def test_singular_gram_is_reported(cb):
    dims = (20, 15, 12)
    X = rand_tensor(dims, torch.float32, 2)
    rng = np.random.default_rng(5)
    f0 = [rng.random((d, 3)).astype(np.float32).astype(np.float64) for d in dims]
    f0[1][:, 2] = 0.0       # a zero column makes Z_S^T Z_S singular
    facs = [torch.tensor(f, device=DEV) for f in f0]
    lam = torch.empty(3, dtype=torch.float64, device=DEV)
    assert cb.cpr_sampled_update(X, dims, lam, facs, 0, 30, seed=1) == cb.ESINGULAR


# ------------------------------------------------------------------------------------------------
# a7: sampled fit, ||X||
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-6), (torch.float64, 1e-12), (torch.bfloat16, 1e-6)])
def test_fit_estimate_and_norm(cb, dtype, tol):
    dims = (33, 40, 27)
    prob = make_problem(dims, 4, C=0.3, eta=0.05, seed=6, dtype=dtype, device=DEV)
    T = to_oracle_array(prob.X, dims)
    rng = np.random.default_rng(7)
    lam0 = rng.uniform(0.2, 0.8, 4)
    fac = [f + 0.01 * rng.standard_normal(f.shape) for f in prob.factors]
    if dtype != torch.float64:
        fac = [f.astype(np.float32).astype(np.float64) for f in fac]
    nrm = cb.cpr_tensor_norm(prob.X, dims)
    assert abs(nrm - np.linalg.norm(T)) < (1e-13 if dtype == torch.float64 else 1e-6) * np.linalg.norm(T)
    fit = cb.cpr_fit_estimate(prob.X, dims, torch.tensor(lam0, device=DEV), [torch.tensor(f, device=DEV) for f in fac],
                              16384, seed=13, b=2)
    idx = streams.fit_sample_indices(13, 2, 16384, dims)
    x = T[tuple(idx[:, m] for m in range(3))]
    ref = cp.sampled_fit(x, lam0, fac, idx, np.linalg.norm(T), T.size)
    assert abs(fit - ref) < tol


# ------------------------------------------------------------------------------------------------
# a0, a9: mixing and unmixing
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims,dtype,tol", [((37, 29, 41), torch.float32, 1e-5), ((130, 64, 65), torch.float32, 1e-5),
                                            ((20, 17, 9, 11), torch.float64, 1e-12),
                                            ((70, 33, 50), torch.bfloat16, 1e-2)])
def test_mix_tensor_matches_oracle(cb, dims, dtype, tol):
    X = rand_tensor(dims, dtype, 8)
    T = to_oracle_array(X, dims)
    Y = cb.cpr_mix_tensor(X, dims, seed=31, b=3)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(31, 3, dims))
    got = to_oracle_array(Y, dims)
    assert rel(got, ref) < tol
    assert abs(np.linalg.norm(got) - np.linalg.norm(T)) < 10 * tol * np.linalg.norm(T)
    # element by element: dense products of length I_n per pass (FP32: split halves, about 2^-21 per
    # product; FP64; BF16: rounded to BF16, 2^-8 relative, after every pass)
    eps = {torch.float32: 2.0 ** -21, torch.float64: 2.0 ** -50, torch.bfloat16: 2.0 ** -8}[dtype]
    depth = len(dims) * (4 * np.sqrt(max(dims)) if dtype != torch.bfloat16 else 4)
    assert_elementwise(got, ref, eps, depth)


def test_unmix_matches_oracle(cb):
    dims = (45, 64, 17)
    rng = np.random.default_rng(9)
    fh = [rng.standard_normal((d, 6)) for d in dims]
    lam = torch.tensor(rng.random(6), device=DEV)
    out_lam, out_f = cb.cpr_unmix_factors(lam, [torch.tensor(f, device=DEV) for f in fh], seed=4, b=1)
    ref = mixing.unmix_factors(fh, mixing.mixing_operators(4, 1, dims))
    for A, Ar in zip(out_f, ref):
        assert rel(A.cpu().numpy(), Ar) < 1e-12
    np.testing.assert_array_equal(out_lam.cpu().numpy(), lam.cpu().numpy())


# ------------------------------------------------------------------------------------------------
# a0-a9: whole runs against the oracle
# ------------------------------------------------------------------------------------------------
def test_cprand_fp64_run_follows_oracle_exactly(cb):
    # plain CPRAND, FP64 50^3, rank-5 N(0,1) factors, 1% noise, R=5, S=80, 50 fixed iterations
    dims = (50, 50, 50)
    prob = make_problem(dims, 5, eta=0.01, seed=1000, dtype=torch.float64, device=DEV, gaussian_factors=True)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(50, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(fixed_iters=50, seed=2000, fit_trace_dev=trace.data_ptr())
    out = cb.cpr_cprand(prob.X, dims, 5, 80, opts=opts)
    ref = cp.cprand(T, 5, 80, seed=2000, rule=cp.StopRule(fixed_iters=50))
    assert out["iters"] == 50 and out["status"] == cb.OK
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-9)
    for A, Ar in zip(out["factors"], ref["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-7


def test_cprand_fp64_stopping_rules_match_oracle(cb):
    dims = (40, 30, 35)
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=17, dtype=torch.float64, device=DEV)
    T = to_oracle_array(prob.X, dims)
    for kw, rule in [({"noise_eta": 0.01}, cp.StopRule(eta=0.01)),
                     ({"stall_iters": 3, "fit_tol": -1.0}, cp.StopRule(tol=-1.0, stall_iters=3)),
                     ({}, cp.StopRule())]:
        opts = cb.cpr_default_opts(seed=5, **kw)
        out = cb.cpr_cprand(prob.X, dims, 4, 60, opts=opts)
        ref = cp.cprand(T, 4, 60, seed=5, rule=rule)
        assert out["iters"] == ref["iters"], (kw, out["iters"], ref["iters"])
        assert abs(out["fit_est"] - ref["fits"][-1]) < 1e-9


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
def test_checkpoint_resume_continues_the_run(cb, dtype, tol):
    # the draws of iteration t depend only on (seed, t, mode, batch index): 10 iterations, then 10
    # more started from the returned factors with the iteration counter continued, give the
    # 20-iteration run (up to the rounding of folding the lazy column scales into the checkpoint)
    dims = (48, 40, 36)
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=19, dtype=dtype, device=DEV)
    tr20 = torch.zeros(20, dtype=torch.float64, device=DEV)
    full = cb.cpr_cprand(prob.X, dims, 4, 60, opts=cb.cpr_default_opts(seed=12, fixed_iters=20,
                                                                       fit_trace_dev=tr20.data_ptr()))
    first = cb.cpr_cprand(prob.X, dims, 4, 60, opts=cb.cpr_default_opts(seed=12, fixed_iters=10))
    tr10 = torch.zeros(10, dtype=torch.float64, device=DEV)
    resumed = cb.cpr_cprand(prob.X, dims, 4, 60, init=first["factors"],
                            opts=cb.cpr_default_opts(seed=12, fixed_iters=10, first_iter=10,
                                                     fit_trace_dev=tr10.data_ptr()))
    assert resumed["iters"] == 10 and resumed["status"] == cb.OK
    np.testing.assert_allclose(tr10.cpu().numpy(), tr20.cpu().numpy()[10:], rtol=0, atol=tol)
    for A, B in zip(resumed["factors"], full["factors"]):
        assert rel(A.cpu().numpy(), B.cpu().numpy()) < tol
    assert rel(resumed["lam"].cpu().numpy(), full["lam"].cpu().numpy()) < tol


def test_repeated_samples_make_square_system_singular(cb):
    # S = R drawn with replacement: a repeated multi-index repeats a row of Z_S, so the sampled
    # least-squares problem is rank deficient and the update must report it rather than solve it
    dims = (80, 70, 90)
    rng = np.random.default_rng(4)
    f0 = [rng.random((d, 64)).astype(np.float32).astype(np.float64) for d in dims]
    idx = streams.ls_sample_indices(77, 1, 5, 0, 64, dims)
    assert len({(a, c) for a, c in zip(idx[:, 1], idx[:, 2])}) < 64     # a repeated row exists
    facs = [torch.tensor(f, device=DEV) for f in f0]
    lam = torch.empty(64, dtype=torch.float64, device=DEV)
    X = rand_tensor(dims, torch.float32, 3)
    assert cb.cpr_sampled_update(X, dims, lam, facs, 0, 64, seed=77, b=1, t=5) == cb.ESINGULAR


@pytest.mark.parametrize("mix", [False, True])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_whole_run_reaches_oracle_fit(cb, mix, dtype):
    # congruence 0.5: both runs reach the noise floor, so the final fits are comparable (with
    # congruence 0.9 the change-in-fit rule stops inside swamps at trajectory-dependent points)
    dims = (60, 50, 40)
    prob = make_problem(dims, 5, C=0.5, eta=0.01, seed=23, dtype=dtype, device=DEV)
    T = to_oracle_array(prob.X, dims)
    S = cp.sample_size(5)
    opts = cb.cpr_default_opts(seed=41, noise_eta=0.01)
    fn = cb.cpr_cprand_mix if mix else cb.cpr_cprand
    out = fn(prob.X, dims, 5, S, opts=opts)
    rule = cp.StopRule(eta=0.01)
    ref = mixing.cprand_mix(T, 5, S, seed=41, rule=rule) if mix else cp.cprand(T, 5, S, seed=41, rule=rule)
    f_gpu = cp.exact_fit(T, out["lam"].cpu().numpy(), [A.cpu().numpy() for A in out["factors"]])
    f_ref = cp.exact_fit(T, ref["lam"], ref["factors"])
    assert out["status"] == cb.OK
    assert abs(f_gpu - f_ref) < 1e-3, (f_gpu, f_ref)


def test_bf16_four_way_run_reaches_oracle_fit(cb):
    # BF16 storage, FP32 accumulation, FP64 R x R work: 4-way, rank 16, congruence 0.5, 1% noise.
    # A fixed 50 outer iterations: this problem has a swamp (the oracle's sampled fit creeps from 0.90
    # to 0.91 over ten iterations), where the change-in-fit rule of Sec. 4.2 fires at a point that
    # depends on the trajectory, and the BF16 rounding of the mixed tensor moves the trajectory
    dims = (40, 36, 32, 30)
    prob = make_problem(dims, 16, C=0.5, eta=0.01, seed=1002, dtype=torch.bfloat16, device=DEV)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(200, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=2002, fixed_iters=50, fit_trace_dev=trace.data_ptr())
    out = cb.cpr_cprand_mix(prob.X, dims, 16, 450, opts=opts)
    ref = mixing.cprand_mix(T, 16, 450, seed=2002, rule=cp.StopRule(fixed_iters=50))
    f_gpu = cp.exact_fit(T, out["lam"].cpu().numpy(), [A.cpu().numpy() for A in out["factors"]])
    f_ref = cp.exact_fit(T, ref["lam"], ref["factors"])
    assert abs(f_gpu - f_ref) < 1e-3, (f_gpu, f_ref, out["iters"], ref["iters"])
    # per iteration: the oracle's CPRAND on the mixed tensor the GPU stored (BF16, so both sides see
    # the same data and the same draws): the traces differ only by the FP32 / FP64 arithmetic -- by
    # 1e-4 at most, or, inside the swamp, where the trajectory amplifies the FP32 rounding of M, by no
    # more than a plain FP32 product with an exact solve moves the oracle's own trace
    Th = to_oracle_array(cb.cpr_mix_tensor(prob.X, dims, seed=2002), dims)
    ref_h = cp.cprand(Th, 16, 450, seed=2002, rule=cp.StopRule(fixed_iters=50))
    err = np.abs(trace.cpu().numpy()[:50] - ref_h["fits"])
    floor = fp32_trace_floor(Th, 16, 450, 2002, 50, ref_h["fits"])
    print("BF16 4-way: per-iteration |dF^| max %.2e, plain FP32 product %.2e" % (err.max(), floor))
    assert np.all(err < max(1e-4, floor)), (err.max(), floor)


@pytest.mark.parametrize("dims", [(24, 30, 100), (20, 12, 1500), (30, 20, 400), (16, 100, 36)])
def test_mix_run_with_compiled_mixing_plans_tracks_oracle(cb, dims):
    # decompositions whose mixing runs the kernels compiled for I_n = 100, 400, 1500 in the last pass
    # (which also writes the mode-N unfolding copy the gathers read) or a middle one, with partial
    # fiber blocks and mode-v extents that are not multiples of 4: sampled-fit trace and factors after
    # a few outer iterations against the oracle
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=77, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(4, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=43, fixed_iters=4, fit_trace_dev=trace.data_ptr())
    out = cb.cpr_cprand_mix(prob.X, dims, 4, 60, opts=opts)
    ref = mixing.cprand_mix(T, 4, 60, seed=43, rule=cp.StopRule(fixed_iters=4))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)
    for A, Ar in zip(out["factors"], ref["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-3


def test_congruence_09_trace_tracks_oracle(cb):
    dims = (60, 50, 40)
    prob = make_problem(dims, 5, C=0.9, eta=0.01, seed=23, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(8, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=41, fixed_iters=8, fit_trace_dev=trace.data_ptr())
    cb.cpr_cprand_mix(prob.X, dims, 5, 80, opts=opts)
    ref = mixing.cprand_mix(T, 5, 80, seed=41, rule=cp.StopRule(fixed_iters=8))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)


@pytest.mark.parametrize("eng", ["auto", "dense"])
def test_full_size_mix_run_tracks_oracle(cb, engine, eng):
    # the 400^3 FP32 workload (R=10, S=230, congruence 0.9), three outer iterations, with the
    # factored-DCT mixing (auto) and with the dense tensor-core mixing
    engine(cb.MIX_AUTO if eng == "auto" else cb.MIX_DENSE)
    dims = (400, 400, 400)
    prob = make_problem(dims, 10, C=0.9, eta=0.01, seed=1001, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    trace = torch.zeros(3, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(fixed_iters=3, seed=2001, fit_trace_dev=trace.data_ptr())
    out = cb.cpr_cprand_mix(prob.X, dims, 10, 230, opts=opts)
    ref = mixing.cprand_mix(T, 10, 230, seed=2001, rule=cp.StopRule(fixed_iters=3))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)
    for A, Ar in zip(out["factors"], ref["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-3


# ------------------------------------------------------------------------------------------------
# a10: batching
# ------------------------------------------------------------------------------------------------
def test_batched_matches_single_runs_and_oracle(cb):
    specs = [((64, 80, 100), 4, 0.0), ((120, 64, 90), 7, 0.5), ((200, 150, 64), 12, 0.9), ((70, 70, 70), 32, 0.3)]
    Xs, dims_l, Rs, Ss, probs = [], [], [], [], []
    for q, (d, R, C) in enumerate(specs):
        p = make_problem(d, R, C=C, eta=0.01, seed=4000 + q, dtype=torch.float32, device=DEV)
        probs.append(p)
        Xs.append(p.X)
        dims_l.append(d)
        Rs.append(R)
        Ss.append(max(R, cp.sample_size(R)))
    opts = [cb.cpr_default_opts(seed=99, batch_index=q, noise_eta=0.01) for q in range(len(specs))]
    outs, _ = cb.cpr_cprand_batched(Xs, dims_l, Rs, Ss, opts, mix=True)
    for q in range(len(specs)):
        T = to_oracle_array(Xs[q], dims_l[q])
        ref = mixing.cprand_mix(T, Rs[q], Ss[q], seed=99, b=q, rule=cp.StopRule(eta=0.01))
        f_gpu = cp.exact_fit(T, outs[q]["lam"].cpu().numpy(), [A.cpu().numpy() for A in outs[q]["factors"]])
        f_ref = cp.exact_fit(T, ref["lam"], ref["factors"])
        assert abs(f_gpu - f_ref) < 1e-3, (q, f_gpu, f_ref)
        single = cb.cpr_cprand_mix(Xs[q], dims_l[q], Rs[q], Ss[q], opts=opts[q])
        f_single = cp.exact_fit(T, single["lam"].cpu().numpy(), [A.cpu().numpy() for A in single["factors"]])
        assert abs(f_gpu - f_single) < 1e-3


# ------------------------------------------------------------------------------------------------
# the three ways of running the iteration loop give the same run
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,mix", [(torch.float64, False), (torch.float32, True), (torch.bfloat16, True)])
def test_loop_paths_agree(cb, dtype, mix):
    dims = (45, 38, 52)
    prob = make_problem(dims, 4, C=0.5, eta=0.01, seed=31, dtype=dtype, device=DEV)
    T = to_oracle_array(prob.X, dims)
    fn = cb.cpr_cprand_mix if mix else cb.cpr_cprand
    runs = {}
    for path in (cb.LOOP_CLUSTER, cb.LOOP_CLUSTER_DIST, cb.LOOP_GRAPH, cb.LOOP_STREAM):
        trace = torch.zeros(12, dtype=torch.float64, device=DEV)
        opts = cb.cpr_default_opts(seed=8, fixed_iters=12, fit_trace_dev=trace.data_ptr(), loop_path=path)
        out = fn(prob.X, dims, 4, 60, opts=opts)
        assert out["iters"] == 12 and out["status"] == cb.OK
        runs[path] = (trace.cpu().numpy(), [A.cpu().numpy() for A in out["factors"]], out["lam"].cpu().numpy())
    if mix:
        # the oracle's CPRAND on the mixed tensor the GPU stored (BF16 storage rounds it), unmixed
        # with the oracle's own operators
        Th = to_oracle_array(cb.cpr_mix_tensor(prob.X, dims, seed=8), dims)
        ops = mixing.mixing_operators(8, 0, dims)
        ref = cp.cprand(Th, 4, 60, seed=8, rule=cp.StopRule(fixed_iters=12))
        ref["factors"] = mixing.unmix_factors(ref["factors"], ops)
    else:
        ref = cp.cprand(T, 4, 60, seed=8, rule=cp.StopRule(fixed_iters=12))
    tol = 1e-9 if dtype == torch.float64 else 1e-4
    for path, (trace, facs, lam) in runs.items():
        np.testing.assert_allclose(trace, ref["fits"], rtol=0, atol=tol)
        for A, Ar in zip(facs, ref["factors"]):
            assert rel(A, Ar) < (1e-7 if dtype == torch.float64 else 1e-3), path


@pytest.mark.parametrize("path", ["cluster", "cluster_dist", "graph"])
def test_ill_conditioned_gram_fp64_matches_oracle(cb, path):
    # congruence 0.9 and R = 32: sampled Grams with condition numbers in the hundreds, where an FP32
    # inverse start is far from FP64 accuracy.  With an FP64 tensor the contraction is FP64, so every
    # error beyond FP64 rounding is the solver's: the FP32 start must be refined (Newton-Schulz steps
    # until the residual bound is below 1e-13) to the oracle's QR solve within 1e-8 after two outer
    # iterations
    dims = (60, 55, 50)
    prob = make_problem(dims, 32, C=0.9, eta=0.01, seed=92, dtype=torch.float64, device=DEV)
    T = to_oracle_array(prob.X, dims)
    lp = {"cluster": cb.LOOP_CLUSTER, "cluster_dist": cb.LOOP_CLUSTER_DIST, "graph": cb.LOOP_GRAPH}[path]
    trace = torch.zeros(2, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=19, fixed_iters=2, fit_trace_dev=trace.data_ptr(), loop_path=lp)
    out = cb.cpr_cprand(prob.X, dims, 32, 1109, opts=opts)
    assert out["status"] == cb.OK
    ref = cp.cprand(T, 32, 1109, seed=19, rule=cp.StopRule(fixed_iters=2))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-10)
    for A, Ar in zip(out["factors"], ref["factors"]):
        assert rel(A.cpu().numpy(), Ar) < 1e-8


@pytest.mark.parametrize("path", ["cluster", "cluster_dist", "grid_tc", "grid_fma"])
def test_ill_conditioned_gram_matches_oracle(cb, path):
    # the same conditioning with an FP32 tensor: here the FP32 rounding of M = X_S Z_S, amplified by
    # the Gram's condition number, moves the factors by more than 1e-4 whatever the solver does (a
    # plain FP32 product with an exact FP64 solve lands 3e-4 to 1.3e-3 from the oracle after two
    # iterations).  Every engine must do no worse than that plain FP32 form (or than 1e-4, the bar of
    # well-conditioned problems), and the sampled fits must agree to 1e-4
    dims = (120, 110, 100)
    prob = make_problem(dims, 32, C=0.9, eta=0.01, seed=91, dtype=torch.float32, device=DEV)
    T = to_oracle_array(prob.X, dims)
    lp = {"cluster": cb.LOOP_CLUSTER, "cluster_dist": cb.LOOP_CLUSTER_DIST, "grid_tc": cb.LOOP_GRID,
          "grid_fma": cb.LOOP_GRID}[path]
    trace = torch.zeros(2, dtype=torch.float64, device=DEV)
    opts = cb.cpr_default_opts(seed=19, fixed_iters=2, fit_trace_dev=trace.data_ptr(), loop_path=lp)
    engine = {"grid_tc": cb.CONTRACT_TC, "grid_fma": cb.CONTRACT_FMA}.get(path, cb.CONTRACT_AUTO)
    prev = cb.cpr_set_contract_engine(engine)
    try:
        out = cb.cpr_cprand(prob.X, dims, 32, 1109, opts=opts)
    finally:
        cb.cpr_set_contract_engine(prev)
    assert out["status"] == cb.OK
    ref = cp.cprand(T, 32, 1109, seed=19, rule=cp.StopRule(fixed_iters=2))
    np.testing.assert_allclose(trace.cpu().numpy(), ref["fits"], rtol=0, atol=1e-4)
    floor = fp32_product_floor(T, 32, 1109, 19, 2, ref)
    errs = [rel(A.cpu().numpy(), Ar) for A, Ar in zip(out["factors"], ref["factors"])]
    print("factor errors", errs, "plain FP32 product", floor)
    for e, f in zip(errs, floor):
        assert e < max(1e-4, f)


def test_cluster_path_rejects_problems_that_do_not_fit(cb):
    dims = (3000, 20, 20)      # 3000 x 64 FP32 partial rows per CTA exceed the cluster's shared memory
    X = rand_tensor(dims, torch.float32, 4)
    opts = cb.cpr_default_opts(seed=1, fixed_iters=1, loop_path=cb.LOOP_CLUSTER)
    with pytest.raises(cb.CprError):
        cb.cpr_cprand(X, dims, 64, 100, opts=opts)


@pytest.mark.parametrize("path", ["cluster", "cluster_dist", "graph"])
@pytest.mark.parametrize("dims", [(41, 37, 29), (13, 11, 9, 7)])
def test_unfolding_copies_give_identical_runs(cb, path, dims):
    # gathering each mode from its column-major unfolding reads the same values in the same order
    prob = make_problem(dims, 3, C=0.5, eta=0.01, seed=77, dtype=torch.float32, device=DEV)
    lp = {"cluster": cb.LOOP_CLUSTER, "cluster_dist": cb.LOOP_CLUSTER_DIST, "graph": cb.LOOP_GRAPH}[path]
    traces = []
    for layout in (0, 1):
        trace = torch.zeros(6, dtype=torch.float64, device=DEV)
        opts = cb.cpr_default_opts(seed=3, fixed_iters=6, fit_trace_dev=trace.data_ptr(), loop_path=lp,
                                   layout=layout)
        out = cb.cpr_cprand_mix(prob.X, dims, 3, 40, opts=opts)
        traces.append((trace.cpu().numpy(), [A.cpu().numpy() for A in out["factors"]]))
    np.testing.assert_array_equal(traces[0][0], traces[1][0])
    for A, B in zip(traces[0][1], traces[1][1]):
        np.testing.assert_array_equal(A, B)


# ------------------------------------------------------------------------------------------------
# a0 on the tensor cores (dense engine): FP32 tensors whose dims are multiples of 4 take the tcgen05
# path (FP16 halves when every dim is a multiple of 8, else 3xTF32; FP32-level accuracy); ragged
# tiles in every direction, several column blocks; other dims the SIMT dense product (37 x 29 x 41)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(64, 48, 40), (132, 20, 36), (300, 12, 8), (516, 8, 12), (16, 12, 20, 8),
                                  (400, 400, 400), (37, 29, 41)])
def test_tensor_core_mixing_matches_oracle(cb, engine, dims):
    engine(cb.MIX_DENSE)
    X = rand_tensor(dims, torch.float32, 11)
    T = to_oracle_array(X, dims)
    Y = cb.cpr_mix_tensor(X, dims, seed=5, b=0)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(5, 0, dims))
    assert rel(to_oracle_array(Y, dims), ref) < 1e-5


# ------------------------------------------------------------------------------------------------
# a0 by the factored DCT-II (mixed-radix FFT per fiber): stages of radix 2 to 25 (plain and
# two-level), one to three stages, orders 2 to 4, fiber blocks that run past the end of a mode, blocks
# of 2 to 32 fibers, the 400^3 and 1500 x ... sizes; the kernels compiled for I_n = 400, 1500 and 100
# with full blocks (vector stores), a partial last block, and a mode-v extent that is not a multiple
# of 4 (scalar stores); mode extents with many blocks and a ragged last one (1500 x 301 x 9,
# 100 x 97 x 61 x 3); FP32 to 1e-6 relative (FP32 FFT rounding), BF16 to the BF16 bar
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(64, 48, 40), (300, 12, 8), (16, 12, 20, 8), (40, 45, 21), (7, 10, 5), (20, 30),
                                  (50, 15, 12, 6), (14, 9, 35), (96, 20, 45), (35, 14, 21), (6000, 8, 5),
                                  (400, 400, 400), (1500, 60, 20), (400, 20, 16), (30, 400, 18), (100, 24, 30),
                                  (24, 100, 17), (12, 1500, 9), (1500, 301, 9), (100, 97, 61, 3)])
def test_fft_mixing_matches_oracle(cb, engine, dims):
    X = rand_tensor(dims, torch.float32, 12)
    T = to_oracle_array(X, dims)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(7, 2, dims))
    Y = cb.cpr_mix_tensor(X, dims, seed=7, b=2)
    got = to_oracle_array(Y, dims)
    assert rel(got, ref) < 1e-6
    # element by element: FP32 butterflies, about 8 log2(I_n) roundings per entry and pass
    assert_elementwise(got, ref, 2.0 ** -23, 8 * len(dims) * np.log2(max(dims)))
    # the dense engine computes the same operator (its split-TF32 error grows with I_n: 1.3e-5 at
    # I_n = 1500, where the FFT's stays below 1e-6)
    engine(cb.MIX_DENSE)
    Yd = cb.cpr_mix_tensor(X, dims, seed=7, b=2)
    gotd = to_oracle_array(Yd, dims)
    assert rel(gotd, ref) < 3e-5
    assert_elementwise(gotd, ref, 2.0 ** -21, 4 * len(dims) * np.sqrt(max(dims)))


# lengths of at least 33 with a prime factor above 7 by Bluestein's chirp-z form (the length-I DFT as
# a cyclic convolution of a 7-smooth length M >= 2 I - 1: 37 -> 75, 53 -> 105, 61 -> 125,
# 127 -> 256, 331 -> 672, 34 -> 70, 38 -> 75, 41 -> 81, 43 -> 90, 509 -> 1024), alone and next to
# 7-smooth modes and to a short one on the dense path (26), with partial blocks; FP32 to 2e-6
# relative, element-wise with the depth of two length-M transforms per pass
@pytest.mark.parametrize("dims", [(61, 37, 53), (127, 12, 10), (331, 24, 9), (26, 34, 38), (41, 43, 30, 7),
                                  (509, 40, 6), (40, 509, 6)])
def test_bluestein_mixing_matches_oracle(cb, dims):
    X = rand_tensor(dims, torch.float32, 13)
    T = to_oracle_array(X, dims)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(7, 2, dims))
    got = to_oracle_array(cb.cpr_mix_tensor(X, dims, seed=7, b=2), dims)
    assert rel(got, ref) < 2e-6
    assert_elementwise(got, ref, 2.0 ** -23, 16 * len(dims) * np.log2(2 * max(dims)))


@pytest.mark.parametrize("dims", [(53, 26, 40), (37, 100, 20)])
def test_bluestein_mixing_bf16_matches_oracle(cb, dims):
    # BF16 in and out (rounded after every mode product), the Bluestein form in FP32 between
    X = rand_tensor(dims, torch.bfloat16, 14)
    T = to_oracle_array(X, dims)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(7, 2, dims))
    got = to_oracle_array(cb.cpr_mix_tensor(X, dims, seed=7, b=2), dims)
    assert rel(got, ref) < 1e-2
    assert_elementwise(got, ref, 2.0 ** -8, 4 * len(dims))


@pytest.mark.parametrize("dims", [(70, 30, 50), (100, 20, 12, 10), (400, 24, 10), (1500, 12, 9)])
def test_fft_mixing_bf16_matches_oracle(cb, dims):
    # BF16 in and out, rounded to BF16 after every mode product (as the dense BF16 engine does)
    X = rand_tensor(dims, torch.bfloat16, 13)
    T = to_oracle_array(X, dims)
    Y = cb.cpr_mix_tensor(X, dims, seed=9, b=0)
    ref = mixing.mix_tensor(T, mixing.mixing_operators(9, 0, dims))
    got = to_oracle_array(Y, dims)
    assert rel(got, ref) < 1e-2
    assert abs(np.linalg.norm(got) - np.linalg.norm(T)) < 1e-2 * np.linalg.norm(T)
    # element by element: each pass rounds every entry to BF16 (half an ulp, 2^-9 relative); the
    # roundings of the earlier passes reach an entry spread at the rms scale
    assert_elementwise(got, ref, 2.0 ** -8, 4 * len(dims))


def test_mix_engine_switch_rejects_unknown_values(cb):
    prev = cb.cpr_set_mix_engine(cb.MIX_AUTO)
    try:
        with pytest.raises(ValueError):
            cb.cpr_set_mix_engine(17)
        assert cb.cpr_set_mix_engine(cb.MIX_DENSE) == cb.MIX_AUTO
        assert cb.cpr_set_mix_engine(cb.MIX_AUTO) == cb.MIX_DENSE
    finally:
        cb.cpr_set_mix_engine(prev)
