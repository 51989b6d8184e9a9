"""Tensor-core band form against the FP64 oracle: Eq. 8 as a direct sum over
the window for the in-band bins, with the operands in BF16, BF16 hi + lo
(three products) or TF32, FP32 accumulation.

Every bar is derived from the arithmetic of the form (no tolerance is tuned
to the result).  With u the unit roundoff of the operand type (BF16 2^-8,
TF32 2^-11) and A_m = sum_j |x[m H + j - M]| |g_j| (A'_m with g'):
  STFT   |V_tc - V| <= c A_m, c = 2.01 u + u^2 + P L 2^-23
         (operand rounding of x and of the basis, P L FP32 accumulations of
         P products; the hi + lo split leaves 3 (2^-16)(1 + 2^-7) per product)
  map    a source whose threshold decision differs sits within its |V| bound
         of the threshold; a destination that differs lies inside the range
         of fine bins reached by the IF estimate's bound, obtained from the
         bounds on V and V' (Eq. 13)
  TFR    each fine bin differs by at most the bounds of the sources both sides
         put there plus the modulus of every source only one side puts there
  inverse |xhat_tc - xhat| <= (2 / Nf) sum_{frames covering p} sum_l |dT| / D[p]
         (Eq. 25, 26: every output sample is a normalised sum of one-sided
         inverse DFTs of the TFR columns) plus the FP32 inverse's own error
The printed statistics are the precision study of the three forms."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import workloads as W

from parity import XHAT_RTOL, as_complex, snr_db

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = ("bf16", "bf16x3", "tf32")


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build_tc()
    S.load_tc()
    return S


def coeff(form: str, L: int) -> float:
    if form == "bf16":
        u, p = 2.0 ** -8, 1
        cin = 2.01 * u + u * u
    elif form == "tf32":
        u, p = 2.0 ** -11, 1
        cin = 2.01 * u + u * u
    else:
        p = 3
        cin = 3 * 2.0 ** -16 * (1 + 2.0 ** -7)
    return cin + p * L * 2.0 ** -23


def frame_abs_sums(x, w, hop, F):
    """sum_j |x[m hop + j - M]| |w_j| for m < F (zero outside the signal)."""
    L = len(w)
    M = (L - 1) // 2
    xp = np.zeros(M + (F - 1) * hop + L + 1)
    n = min(len(x), len(xp) - M)
    xp[M:M + n] = np.abs(x[:n])
    full = np.convolve(xp, np.abs(w)[::-1], mode="valid")
    return full[::hop][:F]


def run_tc(S, params, x32, form):
    plan = S.Plan(**params)
    x = torch.from_numpy(x32).cuda()
    V, Vd = plan.tc_stft(x, form)
    om, dest = plan.tc_reassign_map(x, form)
    tfr = plan.tc_forward(x, form)
    xhat = plan.inverse(tfr)
    q = S.sst_tc_plan_query(plan._tc_handle(form))
    torch.cuda.synchronize()
    out = dict(V=as_complex(V.cpu().numpy()), Vd=as_complex(Vd.cpu().numpy()), omega=om.cpu().numpy(),
               dest=dest.cpu().numpy().astype(np.int64), T=as_complex(tfr.cpu().numpy()),
               xhat=xhat.cpu().numpy().astype(np.float64), hankel=q["hankel_view"])
    plan.close()
    return out


def check_form(g, r, params, x64, form, clean=None):
    L, hop, nf, z = params["L"], params["hop"], params["nfft"], params["z"]
    F, nb = r.V.shape
    nbo = r.T.shape[1]
    gw, dgw = O.window(L, params["sigma"])
    c = coeff(form, L)
    A = np.repeat(frame_abs_sums(x64, gw, hop, F)[:, None], nb, axis=1)
    Ad = np.repeat(frame_abs_sums(x64, dgw, hop, F)[:, None], nb, axis=1)
    vmax = np.abs(r.V).max()
    eV = c * A + 1e-12 * vmax
    eD = c * Ad + 1e-12 * np.abs(r.Vd).max()
    st = {}

    # STFT
    dV, dD = np.abs(g["V"] - r.V), np.abs(g["Vd"] - r.Vd)
    assert np.all(dV <= eV), f"{form}: V outside bound, worst ratio {np.max(dV / eV):.3f}"
    assert np.all(dD <= eD), f"{form}: V' outside bound, worst ratio {np.max(dD / eD):.3f}"
    st["stft_rel"] = dV.max() / vmax
    st["stft_over_A"] = float(np.max(dV / np.maximum(A, 1e-300)))
    st["stft_d_rel"] = dD.max() / np.abs(r.Vd).max()

    # threshold decisions
    aV = np.abs(r.V)
    dgam = params["gamma"] * eV.max() if params["relative"] else 0.0
    keep_o, keep_g = r.dest != -1, g["dest"] != -1
    flip = keep_o != keep_g
    if flip.any():
        assert np.all(np.abs(aV[flip] - r.gamma) <= eV[flip] + dgam + 1e-6 * r.gamma + 1e-7 * vmax), \
            f"{form}: threshold decision differs away from the threshold"
    st["flips"] = int(flip.sum())

    # destinations: the oracle's fractional position u = z (omega - k_lo) + 1/2,
    # widened by z times the IF bound, must reach the CUDA side's bin
    both = keep_o & keep_g
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.abs(r.Vd) / aV
        dq = (eD * aV + np.abs(r.Vd) * eV) / (aV * (aV - eV))
        dom = (nf / (2 * np.pi)) * np.where(aV > eV, dq, np.inf) + 1e-5 * (1 + (nf / (2 * np.pi)) * q)
    u = z * (r.omega - r.k_lo) + 0.5
    lo = np.floor(np.where(np.isfinite(dom), u - z * dom, -1e18))
    hi = np.floor(np.where(np.isfinite(dom), u + z * dom, 1e18))
    dg_ = g["dest"]
    ok_in = (dg_ >= 0) & (dg_ >= lo) & (dg_ <= hi)
    ok_off = (dg_ == -2) & ((lo < 0) | (hi >= nbo))
    diff = both & (dg_ != r.dest)
    bad = diff & ~(ok_in | ok_off)
    assert not bad.any(), f"{form}: destination outside the IF bound at {np.argwhere(bad)[:5]}"
    kept = int((keep_o | keep_g).sum())
    st["map_rate"] = (int(diff.sum()) + st["flips"]) / max(kept, 1)
    st["omega_err_med"] = float(np.median(np.abs(g["omega"] - r.omega)[both]))

    # TFR
    allow = np.zeros((F, nbo))
    rows = np.arange(F)[:, None].repeat(nb, axis=1)
    same = both & (dg_ == r.dest) & (r.dest >= 0)
    np.add.at(allow, (rows[same], r.dest[same]), eV[same])
    moved = (diff | flip)
    mo = moved & (r.dest >= 0)
    np.add.at(allow, (rows[mo], r.dest[mo]), aV[mo] + eV[mo])
    mg = moved & (dg_ >= 0)
    np.add.at(allow, (rows[mg], dg_[mg]), aV[mg] + eV[mg])
    dT = np.abs(g["T"] - r.T)
    assert np.all(dT <= allow + 1e-6 * vmax), f"{form}: TFR outside bound at {np.argwhere(dT > allow + 1e-6 * vmax)[:5]}"
    st["tfr_rel"] = dT.max() / np.abs(r.T).max()

    # inverse
    n = len(x64)
    D = O.normaliser(gw, hop, n)
    E = dT.sum(axis=1)
    M = (L - 1) // 2
    up = np.zeros(F * hop + L)
    up[np.arange(F) * hop] = E
    cover = np.convolve(up, np.ones(L))[M:M + n]
    bound = (2.0 / nf) * cover / D + XHAT_RTOL * np.abs(r.xhat).max()
    dx = np.abs(g["xhat"] - r.xhat)
    assert np.all(dx <= bound), f"{form}: xhat outside bound, worst ratio {np.max(dx / bound):.3f}"
    st["xhat_rel"] = dx.max() / np.abs(r.xhat).max()
    if clean is not None:
        st["snr_tc"], st["snr_oracle"] = snr_db(clean, g["xhat"]), snr_db(clean, r.xhat)
    return st


def oracle_of(params, x32):
    p = params
    return O.sst(x32.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
                 p["z"], p["gamma"], p["relative"], inverse_range=(0, len(x32)))


@pytest.mark.parametrize("form", FORMS)
def test_precision_64k(sst, form):
    """The precision workload (Nf 4096, L 2049, hop 16, the 0-6400 Hz band at
    25.6 kHz: 1025 bins), each form against the oracle."""
    w = W.PRECISION_64K
    noisy, clean = w.signal()
    x32 = noisy.astype(np.float32)
    params = w.params()
    r = oracle_of(params, x32)
    g = run_tc(sst, params, x32, form)
    st = check_form(g, r, params, x32.astype(np.float64), form, clean)
    st["hankel"] = g["hankel"]
    print("precision_64k", form, {k: (f"{v:.3e}" if isinstance(v, float) else v) for k, v in st.items()})


SMALL = [
    # ragged frames / columns, Hankel view (hop 8: 16 bytes per row in BF16)
    dict(n=5003, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=500.0, f_hi=3000.0, z=2, gamma=1e-3,
         relative=True),
    # hop 4: 8 bytes per BF16 row -> explicit frame copy; absolute threshold
    dict(n=3001, fs=2000.0, L=129, sigma=16.0, hop=4, nfft=128, f_lo=100.0, f_hi=900.0, z=1, gamma=0.05,
         relative=False),
    # one bin, odd hop
    dict(n=999, fs=1000.0, L=65, sigma=8.0, hop=5, nfft=64, f_lo=250.0, f_hi=250.0 + 1e-9, z=3, gamma=1e-3,
         relative=True),
    # the chirp / FM workload's parameters on a shorter signal (513 bins)
    dict(n=20000, fs=25600.0, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=12800.0, z=1, gamma=1e-3,
         relative=True),
]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("params", SMALL, ids=[f"n{p['n']}_h{p['hop']}_nf{p['nfft']}" for p in SMALL])
def test_small_cases(sst, params, form):
    gen = np.random.default_rng(params["n"] + 7)
    t = np.arange(params["n"]) / params["fs"]
    mid = 0.5 * (params["f_lo"] + params["f_hi"])
    x = np.cos(2 * np.pi * mid * t + 0.3) + 0.5 * np.cos(2 * np.pi * (0.8 * mid + 40 * t) * t) \
        + 0.3 * gen.standard_normal(params["n"])
    x32 = x.astype(np.float32)
    r = oracle_of(params, x32)
    g = run_tc(sst, params, x32, form)
    st = check_form(g, r, params, x32.astype(np.float64), form)
    print(params["n"], form, g["hankel"], {k: (f"{v:.3e}" if isinstance(v, float) else v) for k, v in st.items()})


def test_tc_plan_errors(sst):
    p = sst.Plan(n=1000, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0, f_hi=500)
    with pytest.raises(sst.SstError) as e:
        sst.sst_tc_plan_create(p.handle, 7)
    assert e.value.status == 1
    x = torch.zeros(999, device="cuda")
    tc = p._tc_handle("bf16")
    with pytest.raises(sst.SstError):
        sst.sst_tc_forward(tc, x, 999, p.new_tfr())
    p.close()


@pytest.mark.parametrize("form", FORMS)
def test_cluster_sizes_identical(sst, form):
    """Sharing the basis tile across a cluster (1, 2 or 4 CTAs) changes only
    where the operands come from: the products and their order are the same,
    so the results are bit-identical."""
    w = W.PRECISION_64K
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    h = plan._tc_handle(form)
    outs = []
    for cl in (1, 2, 4):
        try:
            sst.sst_tc_plan_set_cluster(h, cl)
        except sst.SstError as e:
            assert e.status == 6
            continue
        V, Vd = plan.tc_stft(x, form)
        T = plan.tc_forward(x, form)
        outs.append((cl, V.clone(), Vd.clone(), T.clone()))
    torch.cuda.synchronize()
    assert len(outs) >= 2
    for cl, V, Vd, T in outs[1:]:
        assert torch.equal(V, outs[0][1]) and torch.equal(Vd, outs[0][2]) and torch.equal(T, outs[0][3]), cl
    plan.close()


@pytest.mark.parametrize("form", FORMS)
def test_pair_variant(sst, form):
    """The CTA-pair contraction (tcgen05 cta_group::2, M = 256 across two SMs)
    meets the same derived bounds against the oracle on the precision
    workload."""
    w = W.PRECISION_64K
    noisy, clean = w.signal()
    x32 = noisy.astype(np.float32)
    params = w.params()
    r = oracle_of(params, x32)
    plan = sst.Plan(**params)
    h = plan._tc_handle(form)
    try:
        sst.sst_tc_plan_set_cluster(h, 0)
    except sst.SstError as e:
        assert e.status == 6
        pytest.skip("no CTA pair fits")
    x = torch.from_numpy(x32).cuda()
    V, Vd = plan.tc_stft(x, form)
    om, dest = plan.tc_reassign_map(x, form)
    tfr = plan.tc_forward(x, form)
    xhat = plan.inverse(tfr)
    sst.sst_tc_plan_set_cluster(h, 1)
    V1, _ = plan.tc_stft(x, form)
    torch.cuda.synchronize()
    g = dict(V=as_complex(V.cpu().numpy()), Vd=as_complex(Vd.cpu().numpy()), omega=om.cpu().numpy(),
             dest=dest.cpu().numpy().astype(np.int64), T=as_complex(tfr.cpu().numpy()),
             xhat=xhat.cpu().numpy().astype(np.float64))
    st = check_form(g, r, params, x32.astype(np.float64), form, clean)
    st["same_as_cluster1"] = bool(torch.equal(V, V1))
    print("pair", form, {k: (f"{v:.3e}" if isinstance(v, float) else v) for k, v in st.items()})
    plan.close()


def test_bounded_wait_reports_timeout(sst):
    """A contraction whose operand load is withheld (test hook) gives up its
    bounded waits and reports SST_ETIMEOUT; the context stays usable and the
    next contraction is exact again."""
    p = SMALL[0]
    gen = np.random.default_rng(3)
    x32 = (np.cos(np.arange(p["n"]) * 0.3) + 0.1 * gen.standard_normal(p["n"])).astype(np.float32)
    x = torch.from_numpy(x32).cuda()
    plan = sst.Plan(**p)
    h = plan._tc_handle("bf16x3")
    sst.sst_tc_plan_set_cluster(h, 1)
    V0, _ = plan.tc_stft(x, "bf16x3")
    sst.sst_tc_plan_test_withhold(h)
    V = torch.empty_like(V0)
    Vd = torch.empty_like(V0)
    sst.sst_tc_stft(h, x, plan.n, V, Vd)
    with pytest.raises(sst.SstError) as e:
        sst.sst_tc_check(h)
    assert e.value.status == 5
    V1, _ = plan.tc_stft(x, "bf16x3")       # the hook is one-shot; check passes again
    torch.cuda.synchronize()
    assert torch.equal(V0, V1)
    plan.close()


def tc_sweep_cases():
    from test_gpu_sweep import SHAPES, signal
    return [(i, SHAPES[i], signal) for i in range(3, len(SHAPES), 6)]


@pytest.mark.parametrize("case", tc_sweep_cases(), ids=lambda c: f"shape{c[0]}_nf{c[1]['nfft']}_z{c[1]['z']}")
def test_sweep_shapes_bf16x3(sst, case):
    """Shapes of the plan-shape sweep through the tensor band form (BF16 hi +
    lo), against the oracle with the form's bounds (a plan the form rejects
    is skipped)."""
    i, params, signal = case
    x32 = signal(params, 100 + i)
    r = oracle_of(params, x32)
    try:
        g = run_tc(sst, params, x32, "bf16x3")
    except sst.SstError as e:
        pytest.skip(f"tensor form rejects this plan: {e}")
    st = check_form(g, r, params, x32.astype(np.float64), "bf16x3")
    print(params, {k: (f"{v:.3e}" if isinstance(v, float) else v) for k, v in st.items()})
