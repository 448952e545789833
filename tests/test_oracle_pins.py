"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against an exact
integer evaluation, the cost function the update minimises (Section III-C), a dense
solve of the global quadratic whose block-coordinate minimiser the update is, a closed
form, or an exact invariant of Algorithm 1.
"""
import numpy as np
import pytest

import oracle
from oracle import Params, JACOBI, REDBLACK, RASTER_GS


# --------------------------------------------------------------------------- schedule

def _exact_round_pow(side: int, l: int, n: int) -> int:
    """round(side^(l/n)) in exact integer arithmetic: the m with
    (2m-1)^n < 2^n side^l < (2m+1)^n. A tie would need side^l = ((2m+1)/2)^n, which no
    integer satisfies; the assertion checks that no tie occurred."""
    target = (2 ** n) * side ** l
    m = max(0, int(round(float(side) ** (l / n))))
    # walk to the exact answer from the float estimate
    while (2 * m + 1) ** n <= target:
        m += 1
    while m > 0 and (2 * m - 1) ** n >= target:
        m -= 1
    assert (2 * m + 1) ** n != target and (m == 0 or (2 * m - 1) ** n != target)
    return m


def _exact_levels(w: int, h: int) -> int:
    m = max(w, h)
    return max(1, (m - 1).bit_length())     # ceil(log2 m) for m >= 1


@pytest.mark.parametrize("side_range", [range(1, 2049), range(2049, 8193, 7),
                                        [4320, 7680, 8191, 8192, 16383, 16384, 32767]])
def test_schedule_matches_exact_integer_rounding(side_range):
    # Algorithm 1: n_l = ceil(log2(max(w, h))), w_l = round(w^(l/n_l))
    for side in side_range:
        n = _exact_levels(side, 1)
        assert oracle.num_levels(side, 1) == n
        assert oracle.num_levels(1, side) == n
        for nn in {n, n + 1, max(1, n - 1)}:
            for l in range(1, nn + 1):
                assert oracle._load().oracle_level_side(side, l, nn) == \
                    _exact_round_pow(side, l, nn), (side, l, nn)


def test_schedule_tables_golden():
    # level tables of the three single-image workloads, tests/golden/schedules.txt
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "schedules.txt")
    tables = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, rest = line.split(":")
        w, h = map(int, key.split("x"))
        tables[(w, h)] = [tuple(map(int, t.split(","))) for t in rest.split()]
    assert set(tables) == {(128, 128), (2048, 1536), (7680, 4320)}
    for (w, h), levels in tables.items():
        assert oracle.schedule(w, h) == levels
        n = len(levels)
        for l, (wl, hl, kl) in enumerate(levels, start=1):
            assert wl == _exact_round_pow(w, l, n) and hl == _exact_round_pow(h, l, n)
            assert kl == (10 if (wl <= 32 and hl <= 32) else 2)


def test_iteration_rule_on_elongated_inputs():
    # Section III-D: 10 iterations for "low" resolutions, low meaning 32 x 32; a level
    # counts as low only if it fits in 32 x 32 (both sides), else it gets 2
    for w, h in [(1000, 20), (20, 1000), (3000, 33), (33, 33), (32, 32), (4096, 2)]:
        for wl, hl, kl in oracle.schedule(w, h):
            assert kl == (10 if (wl <= 32 and hl <= 32) else 2), (w, h, wl, hl, kl)
    assert [k for _, _, k in oracle.schedule(1000, 20)].count(2) >= 4


def test_paper_defaults():
    # Section IV-F chooses eps_r = 5e-3 and omega = 0.1; Section III-D: 10 iterations
    # at or below 32 x 32, else 2.
    p = Params()
    assert (p.eps_r, p.omega, p.small_size, p.small_iters, p.big_iters) == \
        (5e-3, 0.1, 32, 10, 2)
    assert p.clamp and p.init == 0.0 and p.order == JACOBI


# ----------------------------------------------------------------------------- resize

def test_resize_identity_and_integer_upsample():
    rng = np.random.default_rng(1)
    img = rng.random((7, 9, 3))
    assert np.array_equal(oracle.resize_nearest(img, 9, 7), img)
    # an integer-factor nearest upsample replicates each pixel into a k x k block
    up = oracle.resize_nearest(img, 27, 14)
    assert np.array_equal(up, np.repeat(np.repeat(img, 2, axis=0), 3, axis=1))


def test_resize_picks_the_nearest_source_centre():
    # brute force: the chosen source pixel's centre is the nearest one to the
    # destination centre mapped into source coordinates (ties cannot occur for the
    # half-integer centres unless the ratio makes them exact; both choices are then
    # at distance 0.5, which the bound allows)
    rng = np.random.default_rng(2)
    for _ in range(200):
        sw, sh = rng.integers(1, 40, 2)
        dw, dh = rng.integers(1, 40, 2)
        idx = np.arange(sw * sh, dtype=np.float64).reshape(sh, sw)
        out = oracle.resize_nearest(idx, dw, dh)
        sy, sx = np.divmod(out.astype(np.int64), sw)
        cx = (np.arange(dw) + 0.5) * sw / dw
        cy = (np.arange(dh) + 0.5) * sh / dh
        assert np.all(np.abs(cx[None, :] - (sx + 0.5)) <= 0.5 + 1e-12)
        assert np.all(np.abs(cy[:, None] - (sy + 0.5)) <= 0.5 + 1e-12)


# --------------------------------------------------------------- per-pixel solve

def _local_cost(g, i, I, a, F, B, eps, omega):
    """The local cost of Section III-C for pixel i = (y, x), all channels,
    with the neighbours' F and B held fixed; g = (F_i[3], B_i[3])."""
    y, x = i
    h, w = a.shape
    cost = 0.0
    for c in range(3):
        cost += (a[y, x] * g[c] + (1 - a[y, x]) * g[3 + c] - I[y, x, c]) ** 2
    for dy, dx in ((0, -1), (0, 1), (-1, 0), (1, 0)):
        yj = min(max(y + dy, 0), h - 1)
        xj = min(max(x + dx, 0), w - 1)
        s = eps + omega * abs(a[y, x] - a[yj, xj])
        for c in range(3):
            cost += s * ((g[c] - F[yj, xj, c]) ** 2 + (g[3 + c] - B[yj, xj, c]) ** 2)
    return cost


def test_update_is_the_minimiser_of_the_local_cost():
    rng = np.random.default_rng(3)
    h, w = 5, 6
    I = rng.random((h, w, 3))
    a = rng.random((h, w))
    a[0, 0], a[2, 3] = 0.0, 1.0
    F = rng.random((h, w, 3))
    B = rng.random((h, w, 3))
    p = Params(clamp=False)
    F1, B1 = oracle.level_iterate(I, a, F, B, 1, p)      # one Jacobi sweep
    for y in range(h):
        for x in range(w):
            g = np.concatenate([F1[y, x], B1[y, x]])
            c0 = _local_cost(g, (y, x), I, a, F, B, p.eps_r, p.omega)
            for k in range(6):
                e = np.zeros(6)
                e[k] = 1e-4
                cp = _local_cost(g + e, (y, x), I, a, F, B, p.eps_r, p.omega)
                cm = _local_cost(g - e, (y, x), I, a, F, B, p.eps_r, p.omega)
                # quadratic: symmetric difference is the gradient, which must vanish
                assert abs(cp - cm) / 2e-4 < 1e-9
                assert cp > c0 and cm > c0


def test_hand_solved_pixel():
    # alpha = 1/2, every neighbour F = B = 1/2 and I = 1/2: A = [[1/4+S, 1/4],
    # [1/4, 1/4+S]], b = (1/4 + S/2)(1, 1); the solution is F = B = 1/2.
    I = np.full((3, 3, 3), 0.5)
    a = np.full((3, 3), 0.5)
    F = np.full((3, 3, 3), 0.5)
    F1, B1 = oracle.level_iterate(I, a, F, F, 1, Params(clamp=False))
    assert np.allclose(F1, 0.5, atol=1e-15) and np.allclose(B1, 0.5, atol=1e-15)


def test_one_pixel_closed_form():
    # 1x1 image: all four clamped neighbours are the pixel itself, so one sweep is a
    # proximal step on (U^T g - I)^2 with weight 4 eps: the error e = U^T g - I shrinks
    # by rho = 4 eps / (|U|^2 + 4 eps) per sweep and the part of g orthogonal to U is
    # kept. From g0: g_t = g0 + U (I - U^T g0) (1 - rho^t) / |U|^2.
    eps = 5e-3
    for al, I0, g0 in [(0.3, (0.2, 0.5, 0.7), 0.1), (0.8, (0.9, 0.1, 0.4), 0.0),
                       (0.0, (0.3, 0.3, 0.3), 0.6), (1.0, (0.6, 0.2, 0.1), 0.25)]:
        U = np.array([al, 1 - al])
        rho = 4 * eps / (U @ U + 4 * eps)
        I = np.array(I0).reshape(1, 1, 3)
        a = np.array([[al]])
        for t in (1, 2, 5, 10, 37):
            F, B = oracle.level_iterate(I, a, np.full((1, 1, 3), g0),
                                        np.full((1, 1, 3), g0), t, Params(clamp=False))
            for c in range(3):
                g = np.array([g0, g0]) + U * (I0[c] - U @ [g0, g0]) * (1 - rho ** t) / (U @ U)
                assert abs(F[0, 0, c] - g[0]) < 1e-13 and abs(B[0, 0, c] - g[1]) < 1e-13
        # the full method on a 1x1 input: one level, 10 sweeps from init
        F, B = oracle.ml(I, a, Params(clamp=False, init=g0))
        for c in range(3):
            g = np.array([g0, g0]) + U * (I0[c] - U @ [g0, g0]) * (1 - rho ** 10) / (U @ U)
            assert abs(F[0, 0, c] - g[0]) < 1e-13 and abs(B[0, 0, c] - g[1]) < 1e-13


# ------------------------------------------------------- global quadratic (dense)

def _dense_minimiser(I, a, eps, omega):
    """argmin of E(F, B) = sum_i sum_c (a_i F_i + (1-a_i) B_i - I_i)^2
    + sum over 4-neighbour edges {i,j} (eps + omega |a_i - a_j|) [(F_i-F_j)^2 + (B_i-B_j)^2],
    assembled edge by edge and solved densely, per channel."""
    h, w = a.shape
    n = h * w
    M = np.zeros((2 * n, 2 * n))
    av = a.reshape(-1)
    for i in range(n):
        M[i, i] += av[i] ** 2
        M[i, n + i] += av[i] * (1 - av[i])
        M[n + i, i] += av[i] * (1 - av[i])
        M[n + i, n + i] += (1 - av[i]) ** 2
    for y in range(h):
        for x in range(w):
            i = y * w + x
            for j in ([y * w + x + 1] if x + 1 < w else []) + \
                     ([(y + 1) * w + x] if y + 1 < h else []):
                s = eps + omega * abs(av[i] - av[j])
                for off in (0, n):
                    M[off + i, off + i] += s
                    M[off + j, off + j] += s
                    M[off + i, off + j] -= s
                    M[off + j, off + i] -= s
    F = np.empty((h, w, 3))
    B = np.empty((h, w, 3))
    for c in range(3):
        Ic = I[..., c].reshape(-1)
        r = np.concatenate([av * Ic, (1 - av) * Ic])
        x = np.linalg.solve(M, r)
        F[..., c] = x[:n].reshape(h, w)
        B[..., c] = x[n:].reshape(h, w)
    return F, B


@pytest.mark.parametrize("order,iters", [(JACOBI, 4000), (REDBLACK, 2500),
                                         (RASTER_GS, 2500)])
@pytest.mark.parametrize("shape", [(5, 7), (6, 7), (1, 9)])
def test_fixed_point_is_the_dense_minimiser(order, iters, shape):
    h, w = shape
    rng = np.random.default_rng(10 + h * w)
    a = rng.random((h, w))
    I = rng.random((h, w, 3))
    Fd, Bd = _dense_minimiser(I, a, 5e-3, 0.1)
    F0 = rng.random((h, w, 3))
    B0 = rng.random((h, w, 3))
    F, B = oracle.level_iterate(I, a, F0, B0, iters, Params(clamp=False, order=order))
    assert np.max(np.abs(F - Fd)) < 1e-9 and np.max(np.abs(B - Bd)) < 1e-9


def test_fixed_point_with_clamp_when_minimiser_is_interior():
    h, w = 6, 5
    rng = np.random.default_rng(77)
    a = 0.2 + 0.6 * rng.random((h, w))
    I = 0.4 + 0.2 * rng.random((h, w, 3))
    Fd, Bd = _dense_minimiser(I, a, 5e-3, 0.1)
    assert Fd.min() > 0 and Fd.max() < 1 and Bd.min() > 0 and Bd.max() < 1
    F, B = oracle.level_iterate(I, a, np.full((h, w, 3), 0.5), np.full((h, w, 3), 0.5),
                                4000, Params())
    assert np.max(np.abs(F - Fd)) < 1e-9 and np.max(np.abs(B - Bd)) < 1e-9


# ------------------------------------------------------------ full-method invariants

def _inputs(h, w, seed, grid=False):
    rng = np.random.default_rng(seed)
    a = rng.random((h, w))
    if grid:
        a = np.round(a * 256) / 256          # 1 - (1 - a) == a exactly
    I = rng.random((h, w, 3))
    return I, a


@pytest.mark.parametrize("order", [JACOBI, REDBLACK, RASTER_GS])
def test_outputs_in_unit_interval(order):
    I, a = _inputs(37, 53, 5)
    F, B = oracle.ml(I, a, Params(order=order))
    assert F.min() >= 0 and F.max() <= 1 and B.min() >= 0 and B.max() <= 1
    # without the clamp the unconstrained solve does leave [0, 1] on these inputs,
    # so the clamp is doing work
    Fu, Bu = oracle.ml(I, a, Params(order=order, clamp=False))
    assert min(Fu.min(), Bu.min()) < 0 or max(Fu.max(), Bu.max()) > 1


def test_alpha_one_gives_zero_background_and_foreground_equal_constant_image():
    # alpha = 1: U = (1, 0), so B only sees its neighbours, which start at 0 and stay 0;
    # F is pulled to I, exactly to c for a constant image I = c.
    h, w = 29, 41
    a = np.ones((h, w))
    I = np.full((h, w, 3), 0.37)
    F, B = oracle.ml(I, a)
    assert np.all(B == 0.0)
    assert np.max(np.abs(F - 0.37)) < 1e-12
    # mirror case alpha = 0
    F, B = oracle.ml(I, np.zeros((h, w)))
    assert np.all(F == 0.0)
    assert np.max(np.abs(B - 0.37)) < 1e-12


@pytest.mark.parametrize("order", [JACOBI, REDBLACK, RASTER_GS])
def test_alpha_one_keeps_the_foreground_within_the_smoothing_bound_of_the_image(order):
    # alpha = 1 on a non-constant image: U = (1, 0) and every edge weight is eps_r
    # (omega |d alpha| = 0), so the 2x2 system is diagonal and each update sets
    # (1 + 4 eps_r) F_i = I_i + eps_r * sum_j F_j (a clamped neighbour being F_i itself).
    # Hence F_i - I_i = eps_r * sum_j (F_j - I_i) / (1 + 4 eps_r), at most
    # 4 eps_r / (1 + 4 eps_r) in size with F and I in [0, 1], after any number of sweeps
    # from any start. B only averages its neighbours and keeps its initial 0. Mirrored
    # for alpha = 0.
    I, _ = _inputs(31, 43, 11)
    p = Params(order=order)
    bound = 4 * p.eps_r / (1 + 4 * p.eps_r)
    F, B = oracle.ml(I, np.ones(I.shape[:2]), p)
    dev = np.abs(F - I).max()
    assert np.all(B == 0.0)
    assert 0 < dev <= bound + 1e-12
    F, B = oracle.ml(I, np.zeros(I.shape[:2]), p)
    assert np.all(F == 0.0)
    assert 0 < np.abs(B - I).max() <= bound + 1e-12


def test_alpha_complement_swaps_foreground_and_background():
    I, a = _inputs(23, 31, 6, grid=True)
    F, B = oracle.ml(I, a)
    F2, B2 = oracle.ml(I, 1.0 - a)
    assert np.array_equal(F2, B) and np.array_equal(B2, F)


@pytest.mark.parametrize("order", [JACOBI, REDBLACK])
def test_transpose_equivariance(order):
    I, a = _inputs(40, 40, 7)
    F, B = oracle.ml(I, a, Params(order=order))
    Ft, Bt = oracle.ml(I.transpose(1, 0, 2), a.T, Params(order=order))
    assert np.max(np.abs(Ft.transpose(1, 0, 2) - F)) < 1e-12
    assert np.max(np.abs(Bt.transpose(1, 0, 2) - B)) < 1e-12


def test_red_black_sweep_updates_even_colour_first():
    # With alpha = 1 the matrix of the 2x2 solve is diagonal (U = (1, 0)) and every edge
    # weight is eps_r, so the background update is the plain mean of the four (clamped)
    # neighbours: B_i <- (B_left + B_right + B_up + B_down) / 4, a clamped neighbour being
    # the pixel's own current value. One red-black sweep on a 3x3 image that starts with
    # B = 1 at (x, y) = (1, 0) and 0 elsewhere, worked by hand:
    #   colour x + y even first: (0,0), (2,0), (1,1) see the 1 once -> 1/4; (0,2), (2,2) -> 0;
    #   then the odd colour: (1,0) <- (1/4 + 1/4 + 1 [itself, clamped above] + 1/4) / 4 = 7/16,
    #   (0,1) <- (0 [itself] + 1/4 + 1/4 + 0) / 4 = 1/8, (2,1) likewise 1/8,
    #   (1,2) <- (0 + 0 + 1/4 + 0 [itself]) / 4 = 1/16.
    # Odd colour first would give [[1/16, 1/4, 1/16], [0, 1/16, 0], [0, 0, 0]] instead.
    a = np.ones((3, 3))
    I = np.zeros((3, 3, 3))
    F0 = np.zeros((3, 3, 3))
    B0 = np.zeros((3, 3, 3))
    B0[0, 1, :] = 1.0
    F, B = oracle.level_iterate(I, a, F0, B0, 1, Params(order=REDBLACK))
    want = np.array([[1 / 4, 7 / 16, 1 / 4], [1 / 8, 1 / 4, 1 / 8], [0.0, 1 / 16, 0.0]])
    assert np.max(np.abs(B - want[:, :, None])) < 1e-12
    assert np.all(F == 0.0)   # I = 0 and F = 0: the foreground stays exactly 0


def test_constant_image_with_constant_init_is_a_fixed_point():
    _, a = _inputs(33, 45, 8)
    I = np.full((33, 45, 3), 0.625)
    F, B = oracle.ml(I, a, Params(init=0.625))
    assert np.max(np.abs(F - 0.625)) < 1e-14 and np.max(np.abs(B - 0.625)) < 1e-14


def test_linear_in_the_image_without_clamp():
    I, a = _inputs(30, 26, 9)
    F, B = oracle.ml(I, a, Params(clamp=False))
    F2, B2 = oracle.ml(0.5 * I, a, Params(clamp=False))
    assert np.max(np.abs(F2 - 0.5 * F)) < 1e-12 and np.max(np.abs(B2 - 0.5 * B)) < 1e-12


def test_levels_follow_algorithm_1():
    # the full method equals its levels run one after another from the pinned pieces:
    # resize I, alpha from full resolution, F, B from the previous level, then k sweeps
    I, a = _inputs(45, 38, 11)
    p = Params()
    F = np.zeros((1, 1, 3))
    B = np.zeros((1, 1, 3))
    for (wl, hl, kl) in oracle.schedule(38, 45):
        Il = oracle.resize_nearest(I, wl, hl)
        al = oracle.resize_nearest(a, wl, hl)
        F = oracle.resize_nearest(F, wl, hl)
        B = oracle.resize_nearest(B, wl, hl)
        F, B = oracle.level_iterate(Il, al, F, B, kl, p)
    Fm, Bm = oracle.ml(I, a, p)
    assert np.array_equal(F, Fm) and np.array_equal(B, Bm)


def test_compositing_residual_small_on_synthetic_matte():
    # the data term drives alpha F + (1 - alpha) B towards I (compositing equation);
    # a statistic, not a tolerance gate
    from paper_2006_14970_gb300 import synth
    s = synth.make_sample(96, 80, 123)
    F, B = oracle.ml(s.I, s.alpha)
    a3 = s.alpha[..., None].astype(np.float64)
    res = np.abs(a3 * F + (1 - a3) * B - s.I)
    frac = (s.alpha > 0) & (s.alpha < 1)
    assert res[frac].mean() < 0.02


def test_composite_closed_forms():
    # alpha = 1 keeps the foreground, alpha = 0 the new background, and a hand-evaluated
    # fractional pixel
    F = np.array([[[0.2, 0.4, 0.6], [0.9, 0.1, 0.5], [1.0, 0.0, 0.25]]])
    Bn = np.array([[[0.7, 0.3, 0.1], [0.0, 1.0, 0.5], [0.5, 0.5, 0.75]]])
    a = np.array([[1.0, 0.0, 0.25]])
    out = oracle.composite(a, F, Bn)
    assert np.array_equal(out[0, 0], F[0, 0]) and np.array_equal(out[0, 1], Bn[0, 1])
    assert np.allclose(out[0, 2], [0.25 * 1.0 + 0.75 * 0.5, 0.75 * 0.5, 0.25 * 0.25 + 0.75 * 0.75],
                       atol=1e-16)


@pytest.mark.parametrize("shape", [(5, 7), (1, 9), (8, 3)])
def test_sparse_minimiser_equals_dense_assembly(shape):
    # the oracle's vectorised sparse system against the edge-by-edge dense assembly above
    pytest.importorskip("scipy.sparse")
    from oracle import minimiser
    h, w = shape
    rng = np.random.default_rng(31 + h * w)
    a = rng.random((h, w))
    I = rng.random((h, w, 3))
    for eps, om in ((5e-3, 0.1), (0.02, 1.0)):
        Fd, Bd = _dense_minimiser(I, a, eps, om)
        Fs, Bs = minimiser.minimiser(I, a, eps, om)
        assert np.abs(Fs - Fd).max() < 1e-10 and np.abs(Bs - Bd).max() < 1e-10
        assert minimiser.gradient_norm(I, a, Fs, Bs, eps, om) < 1e-10


def test_minimiser_is_the_limit_of_the_unclamped_iteration():
    pytest.importorskip("scipy.sparse")
    from oracle import minimiser
    rng = np.random.default_rng(4)
    a = rng.random((9, 11))
    I = rng.random((9, 11, 3))
    Fm, Bm = minimiser.minimiser(I, a)
    F, B = oracle.level_iterate(I, a, np.zeros((9, 11, 3)), np.zeros((9, 11, 3)), 3000,
                                Params(clamp=False, order=REDBLACK))
    assert np.abs(F - Fm).max() < 1e-9 and np.abs(B - Bm).max() < 1e-9
