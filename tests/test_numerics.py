"""Host checks (numpy FP32) of two pieces of the mixed path's compensated
arithmetic, as the kernels state them: the bin index of a float-float arrival
whose low part is not renormalised, and the sum of the gradient over a run of
bins from float-float running sums.  They check the arithmetic, not the CUDA
code; the GPU parity tests compare the kernels with the oracle."""
import numpy as np

f32 = np.float32


def bin_of(uh, ul, n_bins):
    """The bin index and fraction as the kernels form them (all steps FP32)."""
    uh, ul = f32(uh), f32(ul)
    if not uh > f32(-1.0):
        return -1, f32(0.0)
    if not uh < f32(n_bins) + f32(64.0):
        return n_bins, f32(0.0)
    kf = np.floor(uh)
    f = f32(f32(uh - kf) + ul)
    df = np.floor(f)
    kf = f32(kf + df)
    f = f32(f - df)
    k = int(kf)
    if k < 0:
        return -1, f
    if k >= n_bins:
        return n_bins, f
    return k, f


def test_bin_index_of_unnormalised_arrivals_near_2_24():
    """Arrivals near 2^24 bins, where FP32 is spaced by 1 or 2, with low parts up
    to ~9 in magnitude: the bin is floor(uh + ul) of the exact sum, except within
    1e-6 bin of an edge."""
    rng = np.random.default_rng(11)
    N = 1 << 24
    bad = 0
    for _ in range(20000):
        u = float(N) - rng.uniform(-40.0, 400.0)
        uh = f32(u + rng.uniform(-8.0, 8.0))  # an unnormalised high part
        ul = f32(u - float(uh))
        exact = float(uh) + float(ul)
        k, f = bin_of(uh, ul, N)
        want = int(np.floor(exact))
        want = -1 if want < 0 else (N if want >= N else want)
        if abs(exact - round(exact)) < 1e-6:
            continue
        bad += k != want
        if 0 <= k < N:
            assert 0.0 <= f <= 1.0
            assert abs(k + float(f) - exact) < 1e-6
    assert bad == 0


def test_bin_index_matches_a_single_step_adjustment_where_that_holds():
    """For normalised arrivals (|low part| below half a unit of the high part's
    last place, as in the shower's own windows) the floor-based adjustment gives
    the same bin and fraction bits as one step of +-1."""
    rng = np.random.default_rng(12)
    for _ in range(20000):
        u = rng.uniform(-2.0, 5000.0)
        uh = f32(u)
        ul = f32(u - float(uh))
        k, f = bin_of(uh, ul, 4096)
        kf = np.floor(uh)
        g = f32(f32(uh - kf) + ul)
        if g < 0:
            kf, g = f32(kf - f32(1.0)), f32(g + f32(1.0))
        elif g >= 1:
            kf, g = f32(kf + f32(1.0)), f32(g - f32(1.0))
        k1 = int(kf)
        k1 = -1 if k1 < 0 else (4096 if k1 >= 4096 else k1)
        if not f32(uh) > f32(-1.0):
            continue
        assert k == k1
        if 0 <= k < 4096:
            assert f == g


def test_run_sums_from_float_float_prefixes():
    """Sums of a gradient over runs of bins, taken as (h1 - h0) + (l1 - l0) from
    FP64 running sums stored as float-float, are as accurate as the FP64
    difference rounded to FP32, also with a large constant part in the gradient
    (where FP32 running sums lose several digits)."""
    rng = np.random.default_rng(13)
    n = 8192
    for offset in (0.0, 5.0, 300.0):
        g = (rng.normal(size=n) + offset).astype(np.float32)
        S = np.concatenate([[0.0], np.cumsum(g.astype(np.float64))])  # FP64, as the kernel forms them
        h = S.astype(np.float32)
        lo = (S - h.astype(np.float64)).astype(np.float32)
        S32 = np.concatenate([[0.0], np.cumsum(g, dtype=np.float32)]).astype(np.float32)
        worst_ff, worst_32 = 0.0, 0.0
        for _ in range(2000):
            a, b = sorted(rng.integers(0, n, size=2))
            exact = float(np.sum(g[a:b + 1].astype(np.float64)))
            ff = float(f32(f32(h[b + 1] - h[a]) + f32(lo[b + 1] - lo[a])))
            scale = max(abs(exact), 1e-30)
            worst_ff = max(worst_ff, abs(ff - exact) / scale)
            worst_32 = max(worst_32, abs(float(f32(S32[b + 1] - S32[a])) - exact) / scale)
        assert worst_ff <= 2.5e-7, (offset, worst_ff)
        if offset >= 300.0:
            assert worst_32 > 100 * worst_ff  # what the float-float sums avoid
