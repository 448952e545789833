// Tile level pass: K (1 or 2) Jacobi sweeps of one pyramid level in one trip through HBM,
// for levels whose strips fit the tensor-map boxes (the top level and gathered levels up
// to about half the input's width).
//
// Each warp owns a strip of 64 columns (two adjacent pixels per lane, 60 written) and
// walks down its rows. Rows arrive in chunks of four source rows (the nearest-resize rows
// of Algorithm 1) in the warp's slot of shared memory, two or three chunks in flight, each
// tracked by an mbarrier with a bounded wait. Each image (I, alpha, F, B) arrives one of
// two ways: one TMA gather of the chunk's four rows of the strip's source span (layouts
// a tensor map can describe, spans within one box), or asynchronous 4-byte copies by
// every lane of just its own two pixels (spans too wide for a box: levels gathered from
// an input several times wider; rows off the 16-byte grid).
//
// The per-pixel update is the closed-form 2x2 solve of Section III-C,
//   g = (U U^T + S I_2)^{-1} (U I + sum_j s_j [F_j; B_j]),  U = (alpha, 1 - alpha),
// with s_j = eps_r + omega |alpha_i - alpha_j| over the 4-neighbourhood and S = sum s_j,
// clamped to [0, 1] (Algorithm 1). Three choices keep the instruction count per pixel low:
//  - Borders by reflection. A neighbour outside the image is the pixel itself (Algorithm 1
//    clamps coordinates). The halo columns and rows outside the image are loaded as the
//    reflection of the image (column -1 holds column 0, column -2 column 1, row h row
//    h - 1, ...), so the edge to a clamped neighbour has weight eps_r and, after every
//    sweep, the reflected pixel holds the same value as the border pixel (the same terms,
//    summed in another order). No update needs a border case.
//  - Running sums. When row r arrives, its state completes the sums of row r - 1 (the
//    neighbour below) and starts the sums of row r (the data term U I, the neighbour above
//    and the left/right neighbours through warp shuffles), so each sweep keeps one row of
//    state and one row of partial sums in registers instead of three rows.
//  - The matrix of a row depends only on alpha: its inverse is formed once per row (when
//    the weight to the row below is known) and serves both sweeps.
// Pairs of pixels use the packed float32x2 arithmetic of sm_100-class GPUs; the final
// multiply-add of each output is a scalar one with saturation, which is the clamp.
#include "fgml_internal.h"

namespace fgml {

// Set by a wait of this file's kernel that gave up (1). Each translation unit has its own
// error word; read_and_clear_tile_error() is read together with the others by fg_sync.
__device__ int g_tile_error;

namespace {

#include "tile_common.cuh"

// ------------------------------------------------------------------ per-lane state

struct FB {              // F and B of the lane's pixel pair, one float2 per channel
    f2 F[3], B[3];
};

// What a row step hands to the next one. After the step of row r:
struct Carry {
    f2 a;                // alpha of row r
    f2 a1;               // alpha of row r - 1 (compositing epilogue only)
    f2 I[3];             // image of row r; after the row's first step, its data terms
                         // alpha I (DF) and (1 - alpha) I (in DB)
    f2 DB[3];
    float hl, hm, hr;    // row r's horizontal edge weights: left of p0, p0-p1, right of p1
    f2 sh;               // (hl + hm, hm + hr)
    f2 wu;               // row r's edge weights to row r - 1
    FB Q;                // starting state of row r
    FB acc1;             // sweep-1 sums of row r without the row below
    FB P;                // sweep-1 result of row r - 1
    FB acc2;             // sweep-2 sums of row r - 1 without the row below
    f2 mFF, mBB, mFB;    // inverse matrix of row r - 1: [[mFF, -mFB], [-mFB, mBB]]
};

struct Lane {
    int lane;
    int oI0, oI1, oA0, oA1, oS0, oS1;   // byte offsets of the two pixels in a row of the slot
    bool pairs;          // 16-bit, I and alpha by gather of an identity level: p1 follows p0
    bool o0, o1;         // the lane writes p0 / p1
    bool vst;            // paired stores allowed (o0 && o1, outputs' bases aligned for pairs)
    bool odd;            // the output pitch is half a pair off: odd rows start mid-pair
    long long col;       // byte offset of p0 in an output row
};

// Row data from the chunk in shared memory (row j of the slot at `slot`).
template <typename T>
__device__ __forceinline__ void load_row(const PassArgs &p, const Lane &L,
                                         const unsigned char *slot, int j, Carry &c) {
    constexpr int es = (int)sizeof(T);
    const unsigned char *I = slot + j * p.lt_row[0];
    const unsigned char *A = slot + p.lt_off[1] + j * p.lt_row[1];
    const unsigned char *F = slot + p.lt_off[2] + j * p.lt_row[2];
    const unsigned char *B = slot + p.lt_off[3] + j * p.lt_row[3];
    bool done = false;
    if constexpr (sizeof(T) == 2) {
        if (L.pairs) {
            // p0 = (c0, c1, c2), p1 = (c0, c1, c2) in three aligned words; alpha in one
            const uint32_t *w = reinterpret_cast<const uint32_t *>(I + L.oI0);
            const f2 u0 = unpack(w[0], (const T *)nullptr), u1 = unpack(w[1], (const T *)nullptr),
                     u2 = unpack(w[2], (const T *)nullptr);
            c.I[0] = mk(u0.x, u1.y);
            c.I[1] = mk(u0.y, u2.x);
            c.I[2] = mk(u1.x, u2.y);
            c.a = unpack(*reinterpret_cast<const uint32_t *>(A + L.oA0), (const T *)nullptr);
            done = true;
        }
    }
    if (!done) {
        c.a = mk(ldsh<T>(A + L.oA0), ldsh<T>(A + L.oA1));
#pragma unroll
        for (int k = 0; k < 3; ++k) c.I[k] = mk(ldsh<T>(I + L.oI0 + k * es), ldsh<T>(I + L.oI1 + k * es));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.Q.F[k] = mk(ldsh<T>(F + L.oS0 + k * es), ldsh<T>(F + L.oS1 + k * es));
        c.Q.B[k] = mk(ldsh<T>(B + L.oS0 + k * es), ldsh<T>(B + L.oS1 + k * es));
    }
}

// Sums of a row: the data terms (DF = alpha I, DB = (1 - alpha) I), the neighbour above
// (weight wu) and the left/right neighbours of X (shuffles; weights hl/hm/hr of the row).
__device__ __forceinline__ void start_sums(const f2 *DF, const f2 *DB, f2 wu, const FB &up,
                                           const FB &X, float hl, float hm, float hr, FB &acc) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lF = __shfl_up_sync(kMask, X.F[k].y, 1);
        const float rF = __shfl_down_sync(kMask, X.F[k].x, 1);
        const float lB = __shfl_up_sync(kMask, X.B[k].y, 1);
        const float rB = __shfl_down_sync(kMask, X.B[k].x, 1);
        f2 sF = fma2(wu, up.F[k], DF[k]);
        f2 sB = fma2(wu, up.B[k], DB[k]);
        sF.x = fmaf(hl, lF, fmaf(hm, X.F[k].y, sF.x));
        sF.y = fmaf(hm, X.F[k].x, fmaf(hr, rF, sF.y));
        sB.x = fmaf(hl, lB, fmaf(hm, X.B[k].y, sB.x));
        sB.y = fmaf(hm, X.B[k].x, fmaf(hr, rB, sB.y));
        acc.F[k] = sF;
        acc.B[k] = sB;
    }
}

// Adds the neighbour below (weight wd) to a pixel pair's sums of the three channels and
// solves: out = clamp(M acc), M = [[mFF, -mFB], [-mFB, mBB]].
template <bool CLAMP>
__device__ __forceinline__ void finish3(const f2 *aF, const f2 *aB, f2 wd, const f2 *dF, const f2 *dB,
                                        f2 mFF, f2 mBB, f2 mFB, f2 *oF, f2 *oB) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const f2 sF = fma2(wd, dF[k], aF[k]);
        const f2 sB = fma2(wd, dB[k], aB[k]);
        const f2 tF = mul2(mFB, sB);
        const f2 tB = mul2(mFB, sF);
        if (CLAMP) {
            oF[k] = mk(__saturatef(fmaf(mFF.x, sF.x, -tF.x)), __saturatef(fmaf(mFF.y, sF.y, -tF.y)));
            oB[k] = mk(__saturatef(fmaf(mBB.x, sB.x, -tB.x)), __saturatef(fmaf(mBB.y, sB.y, -tB.y)));
        } else {
            oF[k] = mk(fmaf(mFF.x, sF.x, -tF.x), fmaf(mFF.y, sF.y, -tF.y));
            oB[k] = mk(fmaf(mBB.x, sB.x, -tB.x), fmaf(mBB.y, sB.y, -tB.y));
        }
    }
}

template <bool CLAMP>
__device__ __forceinline__ void finish(const FB &acc, f2 wd, const FB &dn, f2 mFF, f2 mBB, f2 mFB,
                                       FB &out) {
    finish3<CLAMP>(acc.F, acc.B, wd, dn.F, dn.B, mFF, mBB, mFB, out.F, out.B);
}

template <typename T>
__device__ __forceinline__ void store_row(const PassArgs &p, const Lane &L, int y, const FB &v) {
    const long long pitch = p.d_pitch * (long long)sizeof(T);
    T *Fr = reinterpret_cast<T *>(static_cast<unsigned char *>(p.Fd) + (long long)y * pitch + L.col);
    T *Br = reinterpret_cast<T *>(static_cast<unsigned char *>(p.Bd) + (long long)y * pitch + L.col);
    if (L.vst && L.odd && (y & 1)) {
        // the row starts half a pair off the pair grid: pairs from the second element on
        st_elem(Fr + 0, v.F[0].x);
        st_pair(Fr + 1, v.F[1].x, v.F[2].x);
        st_pair(Fr + 3, v.F[0].y, v.F[1].y);
        st_elem(Fr + 5, v.F[2].y);
        st_elem(Br + 0, v.B[0].x);
        st_pair(Br + 1, v.B[1].x, v.B[2].x);
        st_pair(Br + 3, v.B[0].y, v.B[1].y);
        st_elem(Br + 5, v.B[2].y);
    } else if (L.vst) {
        st_pair(Fr + 0, v.F[0].x, v.F[1].x);
        st_pair(Fr + 2, v.F[2].x, v.F[0].y);
        st_pair(Fr + 4, v.F[1].y, v.F[2].y);
        st_pair(Br + 0, v.B[0].x, v.B[1].x);
        st_pair(Br + 2, v.B[2].x, v.B[0].y);
        st_pair(Br + 4, v.B[1].y, v.B[2].y);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (L.o0) {
                st_elem(Fr + k, v.F[k].x);
                st_elem(Br + k, v.B[k].x);
            }
            if (L.o1) {
                st_elem(Fr + 3 + k, v.F[k].y);
                st_elem(Br + 3 + k, v.B[k].y);
            }
        }
    }
}

// Compositing epilogue of a row: In = alpha F + (1 - alpha) Bn at the lane's pixels.
template <typename T>
__device__ __forceinline__ void composite_row(const PassArgs &p, const Lane &L, int y, const FB &v,
                                              f2 a) {
    const T *Nr = reinterpret_cast<const T *>(static_cast<const unsigned char *>(p.Bn) +
                                              (long long)y * p.bn_pitch * (long long)sizeof(T) + L.col);
    T *Cr = reinterpret_cast<T *>(static_cast<unsigned char *>(p.In) +
                                  (long long)y * p.in_pitch * (long long)sizeof(T) + L.col);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (L.o0) st_elem(Cr + k, fmaf(a.x, v.F[k].x, (1.f - a.x) * ld_elem(Nr + k)));
        if (L.o1) st_elem(Cr + 3 + k, fmaf(a.y, v.F[k].y, (1.f - a.y) * ld_elem(Nr + 3 + k)));
    }
}

// ------------------------------------------------------------------ one row step

// Stages of a row step (row r arrives; `pv` is the carry of row r - 1, `cu` becomes the
// carry of row r):
//  M: the inverse matrix of row r - 1 (its weight to the row below is now known);
//  S1: sweep 1 of row r - 1 completed with row r (K = 1: stored as output row r - 1);
//  S2: sweep 2 of row r - 2 completed with the sweep-1 result of row r - 1, stored;
//  A2: sweep-2 sums of row r - 1 started;
//  A1: sweep-1 sums of row r started.
enum : int { kM = 1, kS1 = 2, kS2 = 4, kA2 = 8, kA1 = 16, kAll = 31 };

template <typename T, int K, bool CLAMP, bool COMP, int ST>
__device__ __forceinline__ void row_step(const PassArgs &p, const Lane &L, const unsigned char *slot,
                                         int j, int r, int Y1, const Carry &pv, Carry &cu) {
    if (COMP) cu.a1 = pv.a;
    load_row<T>(p, L, slot, j, cu);
    const float eps = p.eps, omega = p.omega;
    const float aR = __shfl_down_sync(kMask, cu.a.x, 1);
    cu.hm = edge(cu.a.x, cu.a.y, eps, omega);
    cu.hr = edge(cu.a.y, aR, eps, omega);
    cu.hl = __shfl_up_sync(kMask, cu.hr, 1);
    cu.sh = mk(cu.hl + cu.hm, cu.hm + cu.hr);
    cu.wu = mk(edge(cu.a.x, pv.a.x, eps, omega), edge(cu.a.y, pv.a.y, eps, omega));
    {
        // the row's data terms, used by both sweeps; cu.I holds alpha I from here on
        const f2 be = mk(1.f - cu.a.x, 1.f - cu.a.y);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cu.DB[k] = mul2(be, cu.I[k]);
            cu.I[k] = mul2(cu.a, cu.I[k]);
        }
    }
    if (ST & kM) invert(pv.a, add2(add2(pv.sh, pv.wu), cu.wu), cu.mFF, cu.mBB, cu.mFB);
    if (ST & kS1) {
        const FB &acc = pv.acc1;
        if (K == 1) {
            FB out;
            finish<CLAMP>(acc, cu.wu, cu.Q, cu.mFF, cu.mBB, cu.mFB, out);
            if (r - 1 < Y1) {
                if (COMP) composite_row<T>(p, L, r - 1, out, pv.a);
                store_row<T>(p, L, r - 1, out);
            }
        } else {
            finish<CLAMP>(acc, cu.wu, cu.Q, cu.mFF, cu.mBB, cu.mFB, cu.P);
        }
    }
    if (K == 2 && (ST & kS2)) {
        FB out;
        finish<CLAMP>(pv.acc2, pv.wu, cu.P, pv.mFF, pv.mBB, pv.mFB, out);
        if (r - 2 < Y1) {
            if (COMP) composite_row<T>(p, L, r - 2, out, pv.a1);
            store_row<T>(p, L, r - 2, out);
        }
    }
    if (K == 2 && (ST & kA2)) start_sums(pv.I, pv.DB, pv.wu, pv.P, cu.P, pv.hl, pv.hm, pv.hr, cu.acc2);
    if (ST & kA1) start_sums(cu.I, cu.DB, cu.wu, pv.Q, cu.Q, cu.hl, cu.hm, cu.hr, cu.acc1);
}

// ------------------------------------------------------------------ the kernel



// One strip (`strip` of the pass) run by the calling warp, with its chunk slots at wbase
// and their mbarriers at bar0 (p.tile_slots of each); `phase` holds the parity each
// mbarrier completes next (bit s for barrier s), carried from strip to strip. False if a
// bounded wait gave up (the device error word is then set). Every chunk the strip fills
// is also taken, so nothing is in flight when it returns.
// LANES: some image arrives by per-lane copies (else all by tensor gather).
template <typename T, int K, bool CLAMP, bool COMP, bool LANES>
__device__ __forceinline__ bool tile_strip(const PassArgs &p, const CUtensorMap *mI,
                                           const CUtensorMap *mA, const CUtensorMap *mF,
                                           const CUtensorMap *mB, int strip,
                                           unsigned char *wbase, uint32_t bar0, uint32_t &phase) {
    const int lane = threadIdx.x & 31;
    constexpr int es = (int)sizeof(T);
    const int slots = p.tile_slots;

    // strip geometry: columns X0 .. X0 + 63 (reflected outside the image), rows R0 ..
    const int xs = strip % p.n_xstrips, ys = strip / p.n_xstrips;
    const int X0 = xs * kW - 2;
    const int Y0 = ys * p.strip_h, Y1 = min(Y0 + p.strip_h, p.h);
    const int R0 = Y0 - K;
    const int nrows = (Y1 - Y0) + 2 * K;
    const int nchunks = (nrows + kChunkRows - 1) / kChunkRows;
    const int xf = min(max(X0, 0), p.w - 1), xl = min(max(X0 + 63, 0), p.w - 1);
    const int x = X0 + 2 * lane;
    const int mx0 = min(max(reflect(x, p.w), xf), xl), mx1 = min(max(reflect(x + 1, p.w), xf), xl);
    const int gi0 = nearest_src(mx0, p.Iw, p.w), gi1 = nearest_src(mx1, p.Iw, p.w);
    const int gs0 = nearest_src(mx0, p.sw, p.w), gs1 = nearest_src(mx1, p.sw, p.w);
    const int giF = nearest_src(xf, p.Iw, p.w), gsF = nearest_src(xf, p.sw, p.w);

    // Per image: byte offsets of the lane's two pixels in a row of the slot. Gathered box
    // rows start at the strip's first source byte rounded down to 16; per-lane copies put
    // the lane's words at lane * (words per lane) * 4 (16-bit values keep their position
    // inside their 4-byte word).
    Lane L;
    {
        L.lane = lane;
        const int cI0 = 3 * gi0 * es, cI1 = 3 * gi1 * es, cA0 = gi0 * es, cA1 = gi1 * es;
        const int cS0 = 3 * gs0 * es, cS1 = 3 * gs1 * es;
        if (!LANES || p.lt_mode[0] == 0) {
            const int b = (3 * giF * es) & ~15;
            L.oI0 = cI0 - b;
            L.oI1 = cI1 - b;
        } else if (es == 4) {
            L.oI0 = lane * 24;
            L.oI1 = lane * 24 + 12;
        } else {
            L.oI0 = lane * 16 + (cI0 & 2);
            L.oI1 = lane * 16 + 8 + (cI1 & 2);
        }
        if (!LANES || p.lt_mode[1] == 0) {
            const int b = (giF * es) & ~15;
            L.oA0 = cA0 - b;
            L.oA1 = cA1 - b;
        } else {
            L.oA0 = lane * 8 + (es == 4 ? 0 : (cA0 & 2));
            L.oA1 = lane * 8 + 4 + (es == 4 ? 0 : (cA1 & 2));
        }
        if (!LANES || p.lt_mode[2] == 0) {
            const int b = (3 * gsF * es) & ~15;
            L.oS0 = cS0 - b;
            L.oS1 = cS1 - b;
        } else if (es == 4) {
            L.oS0 = lane * 24;
            L.oS1 = lane * 24 + 12;
        } else {
            L.oS0 = lane * 16 + (cS0 & 2);
            L.oS1 = lane * 16 + 8 + (cS1 & 2);
        }
        // 16-bit gathered identity levels away from the left and right borders: p1 follows p0
        L.pairs = p.Iw == p.w && X0 >= 0 && X0 + 63 < p.w && (!LANES || (p.lt_mode[0] == 0 && p.lt_mode[1] == 0));
        const bool mid = lane >= 1 && lane <= 30;
        L.o0 = mid && x < p.w;
        L.o1 = mid && x + 1 < p.w;
        L.col = 3LL * max(x, 0) * es;
        const int al = es == 4 ? 7 : 3;
        // pitches are whole elements, so a pitch off the pair grid is off by exactly one element
        L.vst = L.o0 && L.o1 && ((reinterpret_cast<uintptr_t>(p.Fd) | reinterpret_cast<uintptr_t>(p.Bd)) & al) == 0;
        L.odd = ((p.d_pitch * es) & al) != 0;
    }
    // lanes 0..3 issue the gathers of I, alpha, F and B: their map, box x and offset
    const CUtensorMap *map = lane == 0 ? mI : lane == 1 ? mA : lane == 2 ? mF : mB;
    const int limg = min(lane, 3);
    const bool gathers = lane < 4 && (!LANES || p.lt_mode[limg] == 0);
    int bx;
    if (lane == 0) bx = (3 * giF * es) / 16 * (16 / p.tile_uI);
    else if (lane == 1) bx = (giF * es) / 16 * (16 / p.tile_uA);
    else bx = (3 * gsF * es) / 16 * (16 / p.tile_uS);
    const int doff = p.lt_off[limg];

    int fslot = 0, tslot = 0;   // slots of the next chunk to fill and to take
    // Chunk c: rows R0 + 4c .. R0 + 4c + 3 (reflected into the image) into slot c % slots.
    // Lanes 0..7 each find one source row (lanes 0-3 of I and alpha, 4-7 of F and B).
    // With per-lane copies every lane first copies its own pixels' words of the four rows
    // and adds an arrival on the slot's mbarrier that completes when they have landed;
    // then lane 0 arrives, setting the bytes the gathers deliver, and lanes 0..3 issue
    // the gathers.
    auto fill = [&](int c) {
        const int k = lane & 3;
        const int lr = reflect(R0 + kChunkRows * c + k, p.h);
        const int v = lane < 4 ? nearest_src(lr, p.Ih, p.h) : nearest_src(lr, p.sh, p.h);
        const int sel = lane >= 2 ? 4 : 0;
        const int y0 = __shfl_sync(kMask, v, sel + 0), y1 = __shfl_sync(kMask, v, sel + 1);
        const int y2 = __shfl_sync(kMask, v, sel + 2), y3 = __shfl_sync(kMask, v, sel + 3);
        // slots are used in turn: fslot is chunk c's (c % slots, kept without a division)
        const int s = fslot;
        fslot = fslot + 1 == slots ? 0 : fslot + 1;
        (void)c;
        const uint32_t bar = bar0 + 8u * (uint32_t)s;
        const uint32_t sbase = saddr(wbase + s * p.tile_chunk);
        // the slot's previous rows have been read by every lane (the caller synchronised
        // the warp); order those reads before the asynchronous copies that overwrite them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (LANES) {
#pragma unroll
            for (int j = 0; j < kChunkRows; ++j) {
                const int yI = __shfl_sync(kMask, v, j), yS = __shfl_sync(kMask, v, 4 + j);
                if (p.lt_mode[0]) {
                    const unsigned char *row = static_cast<const unsigned char *>(p.I) + (long long)yI * p.I_pitch * es;
                    const uint32_t d = sbase + (uint32_t)(j * p.lt_row[0]);
                    if (es == 4) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            cp_async4(d + lane * 24 + 4 * q, row + 3 * gi0 * es + 4 * q);
                            cp_async4(d + lane * 24 + 12 + 4 * q, row + 3 * gi1 * es + 4 * q);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            cp_async4(d + lane * 16 + 4 * q, row + ((3 * gi0 * es) & ~3) + 4 * q);
                            cp_async4(d + lane * 16 + 8 + 4 * q, row + ((3 * gi1 * es) & ~3) + 4 * q);
                        }
                    }
                }
                if (p.lt_mode[1]) {
                    const unsigned char *row = static_cast<const unsigned char *>(p.A) + (long long)yI * p.A_pitch * es;
                    const uint32_t d = sbase + (uint32_t)(p.lt_off[1] + j * p.lt_row[1]);
                    cp_async4(d + lane * 8, row + ((gi0 * es) & ~3));
                    cp_async4(d + lane * 8 + 4, row + ((gi1 * es) & ~3));
                }
                if (p.lt_mode[2]) {
#pragma unroll
                    for (int img = 2; img < 4; ++img) {
                        const unsigned char *row = static_cast<const unsigned char *>(img == 2 ? p.Fs : p.Bs) +
                                                   (long long)yS * p.s_pitch * es;
                        const uint32_t d = sbase + (uint32_t)(p.lt_off[img] + j * p.lt_row[img]);
                        if (es == 4) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                cp_async4(d + lane * 24 + 4 * q, row + 3 * gs0 * es + 4 * q);
                                cp_async4(d + lane * 24 + 12 + 4 * q, row + 3 * gs1 * es + 4 * q);
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                cp_async4(d + lane * 16 + 4 * q, row + ((3 * gs0 * es) & ~3) + 4 * q);
                                cp_async4(d + lane * 16 + 8 + 4 * q, row + ((3 * gs1 * es) & ~3) + 4 * q);
                            }
                        }
                    }
                }
            }
            // one more pending arrival on the barrier, made when this lane's copies land
            asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
            __syncwarp();
        }
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(bar), "r"((uint32_t)p.tile_tx) : "memory");
        __syncwarp();
        if (gathers) {
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                :: "r"(sbase + (uint32_t)doff), "l"(reinterpret_cast<uint64_t>(map)), "r"(bx), "r"(y0), "r"(y1),
                   "r"(y2), "r"(y3), "r"(bar)
                : "memory");
        }
    };
    // Bounded wait for chunk c; false (and the device error word set) if it gave up.
    auto wait = [&](int c) -> bool {
        const int b = tslot;   // chunk c's slot: chunks are taken in order
        tslot = tslot + 1 == slots ? 0 : tslot + 1;
        (void)c;
        const uint32_t bar = bar0 + 8u * (uint32_t)b;
        const uint32_t par = (phase >> b) & 1u;
        phase ^= 1u << b;
        uint32_t ok = 0;
        for (int i = 0; i < kPolls && !ok; ++i) {
            asm volatile(
                "{\n\t.reg .pred q;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(ok) : "r"(bar), "r"(par), "r"(kHintNs) : "memory");
        }
        return __all_sync(kMask, ok != 0);
    };
    // After a wait gave up: wait (bounded) for the chunks still in flight, then return.
    auto abort = [&](int c_taken, int c_filled) {
        if (lane == 0) atomicExch(&g_tile_error, 1);
        for (int c = c_taken; c < c_filled; ++c) wait(c);
        asm volatile("cp.async.wait_all;" ::: "memory");   // this lane's own copies have landed
    };

    int filled = 0;
    for (; filled < slots && filled < nchunks; ++filled) fill(filled);

    Carry C0, C1;
    // chunk 0: the rows before the first output row
    if (!wait(0)) {
        abort(0, filled);
        return false;
    }
    {
        const unsigned char *slot = wbase;
        row_step<T, K, CLAMP, COMP, 0>(p, L, slot, 0, R0, Y1, C0, C0);   // pv unused
        row_step<T, K, CLAMP, COMP, kA1>(p, L, slot, 1, R0 + 1, Y1, C0, C1);
        if (K == 2) {
            row_step<T, K, CLAMP, COMP, kM | kS1 | kA1>(p, L, slot, 2, R0 + 2, Y1, C1, C0);
            row_step<T, K, CLAMP, COMP, kM | kS1 | kA2 | kA1>(p, L, slot, 3, R0 + 3, Y1, C0, C1);
        } else {
            row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 2, R0 + 2, Y1, C1, C0);
            row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 3, R0 + 3, Y1, C0, C1);
        }
    }
    __syncwarp();
    if (filled < nchunks) fill(filled++);
    int cslot = slots > 1 ? 1 : 0;   // slot of chunk c in the loop below
    for (int c = 1; c < nchunks; ++c) {
        if (!wait(c)) {
            abort(c, filled);
            return false;
        }
        const unsigned char *slot = wbase + cslot * p.tile_chunk;
        cslot = cslot + 1 == slots ? 0 : cslot + 1;
        const int r = R0 + kChunkRows * c;
        row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 0, r, Y1, C1, C0);
        row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 1, r + 1, Y1, C0, C1);
        row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 2, r + 2, Y1, C1, C0);
        row_step<T, K, CLAMP, COMP, kAll>(p, L, slot, 3, r + 3, Y1, C0, C1);
        __syncwarp();
        if (filled < nchunks) fill(filled++);
    }
    return true;
}

template <typename T, int K, bool CLAMP, bool COMP, bool LANES>
__global__ void __launch_bounds__(kWarps * 32, FGML_TILE_BLOCKS) level_tile_kernel(
    const PassArgs p, const __grid_constant__ CUtensorMap mI, const __grid_constant__ CUtensorMap mA,
    const __grid_constant__ CUtensorMap mF, const __grid_constant__ CUtensorMap mB) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_enter();
    const int wib = threadIdx.x >> 5;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (warp >= p.n_warps) return;
    unsigned char *wbase = smem + wib * p.tile_slots * p.tile_chunk;
    const uint32_t bar0 = saddr(smem + kWarps * p.tile_slots * p.tile_chunk) + 8u * (uint32_t)(wib * p.tile_slots);
    init_chunk_barriers(bar0, p.tile_slots);
    uint32_t phase = 0;
    tile_strip<T, K, CLAMP, COMP, LANES>(p, &mI, &mA, &mF, &mB, warp, wbase, bar0, phase);
    pdl_leave();
}

// Work-list batch: one persistent launch runs the level passes of many images. Each warp
// pops (level pass, strip) items in list order; an item first waits (bounded, with
// backoff) until every strip of the pass it reads from has finished, then runs as a strip
// of level_tile_kernel (its pass's tensor maps and chunk layout, its slots in the warp's
// region), then counts itself done. The list holds every pass after the passes it depends
// on, and the grid is no larger than what is resident, so the items an item waits for
// are always running or finished.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool wait_count(const int *c, int need, long long budget_ns) {
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (int i = 0; i < (1 << 26); ++i) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if (v >= need) return true;
        if ((long long)(global_ns() - t0) > budget_ns) return false;
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
    return false;
}

template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kWarps * 32, 2) tile_batch_kernel(
    const BatchDesc *descs, const BatchItem *items, int n_items, int *counters, long long wait_ns,
    int region) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ PassArgs sp[kWarps];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *wbase = smem + wib * region;
    const uint32_t bar0 = saddr(smem + kWarps * region) + 8u * (uint32_t)(wib * kBatchMaxSlots);
    init_chunk_barriers(bar0, kBatchMaxSlots);
    uint32_t phase = 0;   // carried across the items: the barriers are initialised once
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&counters[0], 1);
        idx = __shfl_sync(kMask, idx, 0);
        if (idx >= n_items) break;
        const BatchItem it = items[idx];
        const BatchDesc &d = descs[it.desc];
        const int *src_words = reinterpret_cast<const int *>(&d.a);
        int *dst_words = reinterpret_cast<int *>(&sp[wib]);
        for (int k = lane; k < (int)(sizeof(PassArgs) / sizeof(int)); k += 32) dst_words[k] = src_words[k];
        const int iters = d.iters, dep = d.dep, dep_count = d.dep_count;
        __syncwarp();
        const PassArgs &p = sp[wib];
        if (dep >= 0) {
            int ok = 1;
            if (lane == 0) ok = wait_count(&counters[1 + dep], dep_count, wait_ns) ? 1 : 0;
            ok = __shfl_sync(kMask, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(&g_tile_error, 2);
                break;
            }
            // the previous pass's stores are read next through the asynchronous proxy
            __threadfence();
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        const TileMaps &m = d.maps;
        const bool lanes = p.lt_mode[0] || p.lt_mode[1] || p.lt_mode[2];
        bool ok;
        if (iters == 2) {
            ok = lanes ? tile_strip<T, 2, CLAMP, false, true>(p, &m.I, &m.A, &m.F, &m.B, it.warp, wbase, bar0, phase)
                       : tile_strip<T, 2, CLAMP, false, false>(p, &m.I, &m.A, &m.F, &m.B, it.warp, wbase, bar0, phase);
        } else {
            ok = lanes ? tile_strip<T, 1, CLAMP, false, true>(p, &m.I, &m.A, &m.F, &m.B, it.warp, wbase, bar0, phase)
                       : tile_strip<T, 1, CLAMP, false, false>(p, &m.I, &m.A, &m.F, &m.B, it.warp, wbase, bar0, phase);
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(&counters[1 + it.desc], 1);
        }
    }
}

template <typename T, int K, bool CLAMP, bool COMP, bool LANES>
cudaError_t launch_k(const PassArgs &a, const TileMaps &m, cudaStream_t s, int *blocks_per_sm) {
    const size_t smem = level_tile_smem(a.tile_chunk, a.tile_slots);
    auto *kern = level_tile_kernel<T, K, CLAMP, COMP, LANES>;
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, kWarps * 32, smem);
    const int blocks = (a.n_warps + kWarps - 1) / kWarps;
    return launch_pdl(kern, dim3(blocks), dim3(kWarps * 32), smem, s, a, m.I, m.A, m.F, m.B);
}

template <typename T, int K, bool LANES>
cudaError_t launch_kc(int clamp, const PassArgs &a, const TileMaps &m, cudaStream_t s, int *occ) {
    const bool comp = a.In != nullptr;
    if (clamp)
        return comp ? launch_k<T, K, true, true, LANES>(a, m, s, occ) : launch_k<T, K, true, false, LANES>(a, m, s, occ);
    return comp ? launch_k<T, K, false, true, LANES>(a, m, s, occ) : launch_k<T, K, false, false, LANES>(a, m, s, occ);
}

template <typename T>
cudaError_t launch_t(int iters, int clamp, const PassArgs &a, const TileMaps &m, cudaStream_t s,
                     int *occ) {
    const bool lanes = a.lt_mode[0] || a.lt_mode[1] || a.lt_mode[2] || a.lt_mode[3];
    if (iters == 1) return lanes ? launch_kc<T, 1, true>(clamp, a, m, s, occ) : launch_kc<T, 1, false>(clamp, a, m, s, occ);
    if (iters == 2) return lanes ? launch_kc<T, 2, true>(clamp, a, m, s, occ) : launch_kc<T, 2, false>(clamp, a, m, s, occ);
    return cudaErrorInvalidValue;
}

template <typename T, bool CLAMP>
cudaError_t batch_t(const BatchLaunch &b, cudaStream_t s, int *blocks_per_sm) {
    const size_t smem = tile_batch_smem(b.region);
    cudaError_t e = allow_dynamic_smem(tile_batch_kernel<T, CLAMP>);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tile_batch_kernel<T, CLAMP>,
                                                             kWarps * 32, smem);
    tile_batch_kernel<T, CLAMP><<<b.blocks, kWarps * 32, smem, s>>>(b.descs, b.items, b.n_items,
                                                                   b.counters, b.wait_ns, b.region);
    return cudaGetLastError();
}

}  // namespace

size_t tile_batch_smem(int region) {
    return (size_t)kWarps * (size_t)region + (size_t)kWarps * kBatchMaxSlots * 8;
}

cudaError_t launch_tile_batch(int dtype, int clamp, const BatchLaunch &b, cudaStream_t s,
                              int *blocks_per_sm) {
    switch (dtype) {
        case kF32: return clamp ? batch_t<float, true>(b, s, blocks_per_sm) : batch_t<float, false>(b, s, blocks_per_sm);
        case kBF16:
            return clamp ? batch_t<__nv_bfloat16, true>(b, s, blocks_per_sm)
                         : batch_t<__nv_bfloat16, false>(b, s, blocks_per_sm);
        case kF16: return clamp ? batch_t<__half, true>(b, s, blocks_per_sm) : batch_t<__half, false>(b, s, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t read_and_clear_tile_error(int *code, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(code, g_tile_error, sizeof(int), 0,
                                              cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || !*code) return e;
    const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tile_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

cudaError_t enqueue_tile_error_read(int *dst, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(dst, g_tile_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
}

size_t level_tile_smem(int chunk_bytes, int slots) {
    return (size_t)kWarps * slots * (size_t)chunk_bytes + (size_t)kWarps * slots * 8;
}

cudaError_t launch_level_tile(int dtype, int iters, int clamp, const PassArgs &a,
                              const TileMaps &m, cudaStream_t s, int *blocks_per_sm) {
    switch (dtype) {
        case kF32: return launch_t<float>(iters, clamp, a, m, s, blocks_per_sm);
        case kBF16: return launch_t<__nv_bfloat16>(iters, clamp, a, m, s, blocks_per_sm);
        case kF16: return launch_t<__half>(iters, clamp, a, m, s, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
