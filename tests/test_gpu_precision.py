"""The float-pair arithmetic that carries the mixed mode's extended precision, checked
against exact sums.

The CG's dot products and the refinement's residual b - A x (Sec. 3.1.7) run in
float pairs (hi + lo, error-free transforms on the FP32 pipes) instead of FP64.
These tests run the library's own reduction (flip_dot_f32) and residual
(flip_residual_pairs) on adversarial inputs -- heavy cancellation, an exactly zero
sum, magnitudes spread over 2^+-40 -- and compare with the exactly rounded value
(math.fsum over the FP64 products of FP32 inputs, which are exact; Python
fractions for the residual).  The bounds follow the error analysis of the
algorithms used:

* dot product: each thread's run of m products is Ogita, Rump and Oishi's Dot2
  (TwoProduct by FMA, TwoSum, errors summed in FP32), whose error is at most
  gamma_m^2 sum|x_i y_i| (gamma_m = m u / (1 - m u), u = 2^-24); each later addition
  of two pairs (hi + lo) loses at most 3 u^2 (|a| + |b|), the first one (m + 2) u^2
  (|a| + |b|) because a thread's lo part is not renormalised; L levels of such
  additions lie above a thread (warp, CTA, the CTAs' run and warp); the final
  hi + lo in FP64 adds 2^-53 |sum|.
* residual: at most 16 pair operations, each within 3 u^2 of the magnitudes it
  combines, and the scale's pair within u^2 of the FP64 scale: 64 u^2 (|b| +
  s (cnt |x_c| + sum |x_n|)) per cell.

An FP32-only accumulation, a dropped lo part, or the scale rounded to FP32 misses
these bounds by orders of magnitude (the last case is checked below).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2404_01931_gb300 import flip as F

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _exact_dot(x, y):
    return math.fsum((x.astype(np.float64) * y.astype(np.float64)).tolist())


def _dot_bound(x, y, exact):
    n = x.size
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per = -(-n // sms)
    per = -(-per // 32) * 32
    m = -(-per // 1024) + 1                     # longest run of one thread (rounded up)
    gm = m * U / (1 - m * U)
    levels = 5 + 5 + (-(-sms // 32)) + 5       # warp, CTA, CTAs' run per lane, warp
    s_abs = math.fsum(np.abs(x.astype(np.float64) * y.astype(np.float64)).tolist())
    return (gm * gm + (m + 2) * U * U + 3 * levels * U * U) * s_abs + 2.0 ** -52 * abs(exact)


def _gpu_dot(x, y):
    return F.flip_dot_f32(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())


def _cases():
    rng = np.random.default_rng(7)
    n = 1 << 22
    out = {}
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    out["random"] = (x, y)
    # a ~ -b across CTAs: the second half repeats the first with y negated and
    # perturbed by 2^-20, so the exact sum is ~1e-6 of sum |x y|
    yp = (-(y * np.float32(1.0 + 2.0 ** -20))).astype(np.float32)
    out["cancel_halves"] = (np.concatenate([x, x]), np.concatenate([y, yp]))
    # the same inside each thread: partners 1024 entries apart
    xi = np.empty(2 * n, np.float32)
    yi = np.empty(2 * n, np.float32)
    xb, yb, ypb = x.reshape(-1, 1024), y.reshape(-1, 1024), yp.reshape(-1, 1024)
    xi.reshape(-1, 2, 1024)[:, 0] = xb
    xi.reshape(-1, 2, 1024)[:, 1] = xb
    yi.reshape(-1, 2, 1024)[:, 0] = yb
    yi.reshape(-1, 2, 1024)[:, 1] = ypb
    out["cancel_in_thread"] = (xi, yi)
    # an exactly zero sum
    out["zero_sum"] = (np.concatenate([x, x]), np.concatenate([y, -y]))
    # ill-scaled: magnitudes 2^-40 .. 2^40 on both sides, products over 2^+-80
    ex = rng.integers(-40, 41, n)
    ey = rng.integers(-40, 41, n)
    xs = (rng.uniform(1, 2, n) * np.exp2(ex) * rng.choice([-1, 1], n)).astype(np.float32)
    ys = (rng.uniform(1, 2, n) * np.exp2(ey) * rng.choice([-1, 1], n)).astype(np.float32)
    out["ill_scaled"] = (xs, ys)
    # ill-scaled and cancelling: the large products cancel in pairs, the small
    # ones decide the sum
    out["ill_scaled_cancel"] = (np.concatenate([xs, xs]), np.concatenate([ys, -ys * np.float32(
        1.0 + 2.0 ** -22)]).astype(np.float32))
    return out


@pytest.mark.parametrize("case", ["random", "cancel_halves", "cancel_in_thread", "zero_sum",
                                  "ill_scaled", "ill_scaled_cancel"])
def test_dot_product_within_the_float_pair_bound(case):
    x, y = _cases()[case]
    exact = _exact_dot(x, y)
    got = _gpu_dot(x, y)
    bound = _dot_bound(x, y, exact)
    err = abs(got - exact)
    s_abs = math.fsum(np.abs(x.astype(np.float64) * y.astype(np.float64)).tolist())
    fp32 = float(np.dot(x, y))  # numpy's float32 dot, for scale in the message
    assert err <= bound, (f"{case}: |dot - exact| = {err:.3e} > bound {bound:.3e} "
                          f"(sum|xy| = {s_abs:.3e}, exact {exact:.6e}, FP32 dot error "
                          f"{abs(fp32 - exact):.3e})")
    # the bound is ~1e-11 of sum |x y|: a plain FP32 sum would be off by ~1e-4 of it
    assert bound <= 1e-10 * s_abs + 2.0 ** -52 * abs(exact)


def test_dot_product_edge_sizes():
    """Empty input, one entry, and a ragged length that leaves most CTAs idle."""
    assert F.flip_dot_f32(torch.zeros(0, device="cuda"), torch.zeros(0, device="cuda")) == 0.0
    a = torch.tensor([3.0], device="cuda")
    b = torch.tensor([-0.5], device="cuda")
    assert F.flip_dot_f32(a, b) == -1.5
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1037).astype(np.float32)
    y = rng.standard_normal(1037).astype(np.float32)
    exact = _exact_dot(x, y)
    assert abs(_gpu_dot(x, y) - exact) <= _dot_bound(x, y, exact)


# ------------------------------------------------------------------ residual

def _pair(v64):
    """The float pair (hi, lo) nearest a float64 array: hi = fl32(v), lo = fl32(v - hi)."""
    hi = v64.astype(np.float32)
    lo = (v64 - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _residual_case(n=(24, 20, 16), seed=5, perturb=1e-9):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    p = F.default_params(nx, ny, nz)
    s64 = p.dt / (p.rho * p.dx * p.dx)
    t = (rng.uniform(size=nx * ny * nz) < 0.6).astype(np.uint8)
    t[0] = 0  # at least one air cell
    # x: smooth plus noise, as a float pair with a non-trivial lo part
    i = np.arange(nx * ny * nz)
    ci, cj, ck = i % nx, (i // nx) % ny, i // (nx * ny)
    x64 = 1e3 * (1 + 0.01 * np.sin(ci) * np.cos(cj) + 1e-3 * ck) + rng.uniform(-1, 1, i.size)
    xh, xl = _pair(x64 + rng.uniform(-1, 1, i.size) * 2.0 ** -30 * np.abs(x64))
    # b: nearly s A x, so the residual cancels all but ~perturb of it
    ax = _apply_a_f64(t, xh.astype(np.float64) + xl.astype(np.float64), n, s64)
    bh, bl = _pair(ax * (1 + perturb * rng.uniform(-1, 1, i.size)))
    return p, s64, t, (xh, xl), (bh, bl)


def _neighbours(c, n):
    """(inside the grid, index) of the six neighbours of cell c, in the solver's order."""
    nx, ny, nz = n
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    return ((i > 0, c - 1), (i < nx - 1, c + 1), (j > 0, c - nx), (j < ny - 1, c + nx),
            (k > 0, c - nx * ny), (k < nz - 1, c + nx * ny))


def _apply_a_f64(t, x, n, s):
    """s A x in FP64 (7-point row: s (cnt x_c - sum of fluid neighbours' x))."""
    out = np.zeros_like(x)
    for c in np.flatnonzero(t == 1):
        nb = _neighbours(c, n)
        cnt = sum(ok for ok, _ in nb)
        out[c] = s * (cnt * x[c] - sum(x[q] for ok, q in nb if ok and t[q] == 1))
    return out


def _exact_residual(t, x, b, n, s64):
    """(r, T) per fluid cell as Fractions: r = b - s A x exactly, T = |b| + s (cnt |x_c| +
    sum over fluid neighbours |x_n|)."""
    S = Fraction(s64)
    xf = [Fraction(float(h)) + Fraction(float(l)) for h, l in zip(*x)]
    out = {}
    for c in np.flatnonzero(t == 1):
        bc = Fraction(float(b[0][c])) + Fraction(float(b[1][c]))
        cnt, acc, mag = 0, Fraction(0), Fraction(0)
        for ok, q in _neighbours(c, n):
            if not ok:
                continue
            cnt += 1
            if t[q] == 1:
                acc += xf[q]
                mag += abs(xf[q])
        ax = S * (cnt * xf[c] - acc)
        out[c] = (bc - ax, abs(bc) + S * (cnt * abs(xf[c]) + mag))
    return out


def _gpu_residual(p, t, x, b):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rh = torch.empty(t.size, dtype=torch.float32, device="cuda")
    rl = torch.empty_like(rh)
    F.flip_residual_pairs(p, d(t), d(x[0]), d(x[1]), d(b[0]), d(b[1]), rh, rl)
    return rh.cpu().numpy(), rl.cpu().numpy()


@pytest.mark.parametrize("perturb", [1e-9, 0.0, 1e-4])
def test_refinement_residual_within_the_float_pair_bound(perturb):
    n = (24, 20, 16)
    p, s64, t, x, b = _residual_case(n, perturb=perturb)
    rh, rl = _gpu_residual(p, t, x, b)
    ref = _exact_residual(t, x, b, n, s64)
    worst = 0.0
    for c, (r, mag) in ref.items():
        got = Fraction(float(rh[c])) + Fraction(float(rl[c]))
        ratio = float(abs(got - r) / (mag * Fraction(U) ** 2))
        worst = max(worst, ratio)
    assert worst <= 64.0, f"residual error {worst:.1f} u^2 of its magnitudes (bound 64)"
    assert np.all(rh[t != 1] == 0) and np.all(rl[t != 1] == 0)


def test_fp32_scale_would_miss_the_bound():
    """The bound is tight enough to matter: the residual with the operator's scale
    rounded to FP32 (the pair's lo part of s dropped) misses it by orders of magnitude,
    so the pair scale the library uses is what the test pins."""
    n = (24, 20, 16)
    p, s64, t, x, b = _residual_case(n, perturb=0.0)
    ref = _exact_residual(t, x, b, n, float(np.float32(s64)))
    exact = _exact_residual(t, x, b, n, s64)
    worst = max(float(abs(ref[c][0] - exact[c][0]) / (exact[c][1] * Fraction(U) ** 2))
                for c in exact)
    assert worst > 1e3
