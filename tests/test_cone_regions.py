"""The region rule of the small-level launch (csrc/cone.cu, cone_regions in fgml_internal.h),
checked on the CPU: a block that computes every level of a run only on the cells its
output tile depends on — the tile expanded by each level's sweep count (clipped at the
level's borders, where the clamped neighbour is the cell itself), mapped to the level below
by the nearest-resize rule of Algorithm 1 — and that shrinks its valid region by one cell per
sweep on every side not at a border, reproduces the level-by-level Jacobi result exactly.
Every neighbour and every resize source it reads must lie inside the region valid at that
moment (the device kernel's index bounds). Pure Python in float64 with one update
function for both schedules, so equality is exact."""
import numpy as np
import pytest

TW, TH = 32, 16   # the kernel's output tile (kConeTW x kConeTH)


def nsrc(d, S, D):
    return ((2 * d + 1) * S) // (2 * D)


def update(x, y, w, h, A, I, state, eps=5e-3, om=0.1):
    # one clamped Jacobi update of Section III-C at (x, y); state(nx, ny) -> 6 values
    ai = A[y, x]
    S, acc = 0.0, np.zeros(6)
    for nx, ny in ((max(x - 1, 0), y), (min(x + 1, w - 1), y), (x, max(y - 1, 0)), (x, min(y + 1, h - 1))):
        d = eps + om * abs(ai - A[ny, nx])
        S += d
        acc += d * state(nx, ny)
    be = 1 - ai
    a00, a11, a01 = ai * ai + S, be * be + S, ai * be
    m = 1 / (a00 * a11 - a01 * a01)
    out = np.zeros(6)
    for c in range(3):
        bF, bB = ai * I[y, x, c] + acc[c], be * I[y, x, c] + acc[3 + c]
        out[c] = min(1, max(0, (a11 * bF - a01 * bB) * m))
        out[3 + c] = min(1, max(0, (a00 * bB - a01 * bF) * m))
    return out


def gathered(Ifull, Afull, w, h):
    H, W = Afull.shape
    ys = [nsrc(y, H, h) for y in range(h)]
    xs = [nsrc(x, W, w) for x in range(w)]
    return Ifull[np.ix_(ys, xs)], Afull[np.ix_(ys, xs)]


def level_by_level(levels, X0, Ifull, Afull):
    X = X0
    for (w, h, k) in levels:
        ph, pw = X.shape[:2]
        I, A = gathered(Ifull, Afull, w, h)
        S = np.array([[X[nsrc(y, ph, h), nsrc(x, pw, w)] for x in range(w)] for y in range(h)])
        for _ in range(k):
            S = np.array([[update(x, y, w, h, A, I, lambda nx, ny, S=S: S[ny, nx]) for x in range(w)]
                          for y in range(h)])
        X = S
    return X


def by_cones(levels, X0, Ifull, Afull):
    wL, hL = levels[-1][:2]
    ph0, pw0 = X0.shape[:2]
    out = np.full((hL, wL, 6), np.nan)
    for by in range((hL + TH - 1) // TH):
        for bx in range((wL + TW - 1) // TW):
            R = [bx * TW, by * TH, min(bx * TW + TW - 1, wL - 1), min(by * TH + TH - 1, hL - 1)]
            E = [None] * len(levels)
            for l in range(len(levels) - 1, -1, -1):
                w, h, k = levels[l]
                E[l] = [max(R[0] - k, 0), max(R[1] - k, 0), min(R[2] + k, w - 1), min(R[3] + k, h - 1)]
                pw, ph = (levels[l - 1][0], levels[l - 1][1]) if l else (pw0, ph0)
                R = [nsrc(E[l][0], pw, w), nsrc(E[l][1], ph, h), nsrc(E[l][2], pw, w), nsrc(E[l][3], ph, h)]
            P = {(x, y): X0[y, x] for y in range(R[1], R[3] + 1) for x in range(R[0], R[2] + 1)}
            V = R
            for l, (w, h, k) in enumerate(levels):
                e = E[l]
                pw, ph = (levels[l - 1][0], levels[l - 1][1]) if l else (pw0, ph0)
                I, A = gathered(Ifull, Afull, w, h)
                S = {}
                for y in range(e[1], e[3] + 1):
                    for x in range(e[0], e[2] + 1):
                        sx, sy = nsrc(x, pw, w), nsrc(y, ph, h)
                        assert V[0] <= sx <= V[2] and V[1] <= sy <= V[3], "resize source outside the valid region"
                        S[(x, y)] = P[(sx, sy)]
                v = e
                for _ in range(k):
                    nv = [v[0] + (v[0] > 0), v[1] + (v[1] > 0), v[2] - (v[2] < w - 1), v[3] - (v[3] < h - 1)]

                    def get(nx, ny, v=v, S=S):
                        assert v[0] <= nx <= v[2] and v[1] <= ny <= v[3], "neighbour outside the valid region"
                        return S[(nx, ny)]
                    S = {(x, y): update(x, y, w, h, A, I, get)
                         for y in range(nv[1], nv[3] + 1) for x in range(nv[0], nv[2] + 1)}
                    v = nv
                P, V = S, v
            for y in range(by * TH, min(by * TH + TH, hL)):
                for x in range(bx * TW, min(bx * TW + TW, wL)):
                    out[y, x] = P[(x, y)]
    return out


@pytest.mark.parametrize("levels,coarse,full", [
    ([(43, 31, 2), (80, 55, 2), (150, 97, 2)], (23, 17), (150, 97)),   # a run ending at the top
    ([(31, 43, 2), (55, 80, 2)], (17, 23), (97, 150)),                  # taller than wide
    ([(71, 41, 3), (130, 70, 3)], (38, 22), (130, 70)),                 # three sweeps per level
    ([(47, 33, 1), (90, 60, 1)], (25, 17), (90, 60)),                   # one sweep per level
    ([(300, 7, 2)], (152, 4), (300, 7)),                                # thinner than a tile
])
def test_dependency_cones_reproduce_level_by_level_jacobi(levels, coarse, full):
    rng = np.random.default_rng(len(levels) * 1000 + full[0])
    X0 = rng.random((coarse[1], coarse[0], 6))
    Ifull = rng.random((full[1], full[0], 3))
    Afull = rng.random((full[1], full[0]))
    np.testing.assert_array_equal(by_cones(levels, X0, Ifull, Afull), level_by_level(levels, X0, Ifull, Afull))
