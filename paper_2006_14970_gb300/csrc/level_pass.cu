// Level pass: K Jacobi sweeps of one pyramid level in a single trip through HBM.
//
// Each warp owns a strip of 64 columns (two adjacent pixels per lane) and walks down
// its rows. Row r of the starting state is read from HBM exactly once (alpha and I by
// nearest resize of the full-resolution input, F and B by nearest resize of the
// previous level, Algorithm 1); sweep 1 is computed one row behind the loads and sweep 2
// one row behind sweep 1, all in registers: three-row register queues per sweep, left
// and right neighbours through warp shuffles. The two outermost columns of the strip
// are halo, so a warp writes 60 columns; the strip's vertical halo is K rows.
//
// Rows reach the warp in one of two ways:
//  - ring variant (the fast path): a per-warp ring of kRingSlots row slots in shared
//    memory, filled by bulk asynchronous copies (the TMA engine, one elected lane, one
//    copy per image segment) that run several rows ahead; completion is tracked by one
//    mbarrier per slot, and every wait is bounded;
//  - register variant: plain loads one row ahead into registers (used when a strip's
//    source span is too wide for the ring, and for zero-sweep levels).
//
// The per-pixel update is the closed-form 2x2 solve of Section III-C,
//   g = (U U^T + S I_2)^{-1} (U I + sum_j s_j [F_j; B_j]),  U = (alpha, 1 - alpha),
// with s_j = eps_r + omega |alpha_i - alpha_j| over the 4-neighbourhood and S = sum s_j,
// solved through the adjugate and clamped to [0, 1] (Algorithm 1). A neighbour outside
// the image is the pixel itself (Algorithm 1 clamps coordinates): its weight is eps_r
// and its value the pixel's own previous value. The matrix depends only on alpha, so its
// inverse is formed once per row and used by both sweeps. Pairs of pixels use the packed
// float32x2 arithmetic of sm_100-class GPUs.
#include "fgml_internal.h"

#include <algorithm>

namespace fgml {

// Set by a kernel whose bounded wait gave up (1 = an mbarrier wait timed out).
__device__ int g_device_error;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 60;          // output columns per warp
constexpr int kWarpsPerBlock = 4;
constexpr int kLaneCols = 64;        // columns held by a warp (2 per lane)
constexpr int kWaitPolls = 1 << 20;          // try_wait polls before a wait gives up
constexpr uint32_t kWaitHintNs = 2000;       // suspend-time hint of one poll
constexpr int kTileRows = 4;                 // rows per tensor-copy chunk (gather mode: 4)
#ifndef FGML_RING_MIN_BLOCKS
#define FGML_RING_MIN_BLOCKS 2
#endif
constexpr int kRingMinBlocks = FGML_RING_MIN_BLOCKS;   // resident blocks per SM targeted

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return f2(-a.x, -a.y); }

struct FB {                 // F and B of a lane's pixel pair, one float2 per channel
    float2 F[3], B[3];
};

struct RowK {               // per-row data of a lane's pixel pair
    float2 a;               // alpha
    float2 I[3];            // image
    float2 wl, wr, wu, wd;  // weights of the left/right/up/down neighbour, 0 if clamped
    float2 ws;              // eps_r per clamped neighbour (weight of the pixel's own value)
    float2 mFF, mBB, nFB;   // A^{-1} = [[mFF, -nFB'], ...]: F' = mFF bF + nFB bB etc.
};

struct Raw {                // one row as read
    float a0, a1;
    float i0[3], i1[3];
    float f0[3], f1[3], b0[3], b1[3];
};

struct LaneGeo {
    int x;                  // column of the lane's first pixel (may be outside the image)
    int gi0, gi1;           // source columns of the two pixels in I and alpha
    int gs0, gs1;           // source columns in the starting F and B
    bool inL0, inR0, inR1;  // left of p0, right of p0, right of p1 lie inside the image
};

__device__ __forceinline__ float edge_w(float ai, float aj, float eps, float omega) {
    return fmaf(omega, fabsf(ai - aj), eps);
}

// Row r arrives: alpha, I, the starting F/B, and the weights that row r alone fixes.
__device__ __forceinline__ void make_row(const Raw &raw, const LaneGeo &g, int r,
                                         const RowK &above, float eps, float omega,
                                         RowK &k, FB &q) {
    k.a = f2(raw.a0, raw.a1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        k.I[c] = f2(raw.i0[c], raw.i1[c]);
        q.F[c] = f2(raw.f0[c], raw.f1[c]);
        q.B[c] = f2(raw.b0[c], raw.b1[c]);
    }
    const float aL = __shfl_up_sync(kFull, raw.a1, 1);     // left of p0: lane-1's p1
    const float aR = __shfl_down_sync(kFull, raw.a0, 1);   // right of p1: lane+1's p0
    const float e0 = edge_w(raw.a0, aL, eps, omega);
    const float e1 = edge_w(raw.a0, raw.a1, eps, omega);
    const float e2 = edge_w(raw.a1, aR, eps, omega);
    k.wl = f2(g.inL0 ? e0 : 0.f, e1);
    k.wr = f2(g.inR0 ? e1 : 0.f, g.inR1 ? e2 : 0.f);
    float s0 = (g.inL0 ? 0.f : eps) + (g.inR0 ? 0.f : eps);
    float s1 = g.inR1 ? 0.f : eps;
    if (r > 0) {
        k.wu = f2(edge_w(raw.a0, above.a.x, eps, omega), edge_w(raw.a1, above.a.y, eps, omega));
    } else {
        k.wu = f2(0.f, 0.f);
        s0 += eps;
        s1 += eps;
    }
    k.ws = f2(s0, s1);
    k.wd = f2(0.f, 0.f);
}

// Row q's weights are complete (its down weight is known): form A^{-1} once.
// A = [[alpha^2 + S, alpha(1-alpha)], [alpha(1-alpha), (1-alpha)^2 + S]].
__device__ __forceinline__ void finish_row(RowK &k) {
    const float2 S = add2(add2(add2(k.wl, k.wr), add2(k.wu, k.wd)), k.ws);
    const float2 be = f2(1.f - k.a.x, 1.f - k.a.y);
    const float2 A00 = fma2(k.a, k.a, S);
    const float2 A11 = fma2(be, be, S);
    const float2 A01 = mul2(k.a, be);
    const float2 det = fma2(A00, A11, neg2(mul2(A01, A01)));
    const float2 m = f2(__fdividef(1.f, det.x), __fdividef(1.f, det.y));
    k.mFF = mul2(A11, m);
    k.mBB = mul2(A00, m);
    k.nFB = neg2(mul2(A01, m));
}

// One Jacobi update of a row: c = the row's previous state, up/dn = the previous state
// of the rows above and below (ignored where the weight is 0).
template <bool CLAMP>
__device__ __forceinline__ void update(const RowK &k, const FB &c, const FB &up, const FB &dn,
                                       FB &out) {
    const float2 be = f2(1.f - k.a.x, 1.f - k.a.y);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float lF = __shfl_up_sync(kFull, c.F[ch].y, 1);
        const float rF = __shfl_down_sync(kFull, c.F[ch].x, 1);
        const float lB = __shfl_up_sync(kFull, c.B[ch].y, 1);
        const float rB = __shfl_down_sync(kFull, c.B[ch].x, 1);
        // vertical and own terms packed over the pixel pair; the horizontal ones, whose
        // operands straddle lanes, as scalar multiply-adds (no register pairing moves)
        float2 sF = fma2(k.wd, dn.F[ch], fma2(k.ws, c.F[ch], mul2(k.wu, up.F[ch])));
        sF.x = fmaf(k.wl.x, lF, fmaf(k.wr.x, c.F[ch].y, sF.x));
        sF.y = fmaf(k.wl.y, c.F[ch].x, fmaf(k.wr.y, rF, sF.y));
        float2 sB = fma2(k.wd, dn.B[ch], fma2(k.ws, c.B[ch], mul2(k.wu, up.B[ch])));
        sB.x = fmaf(k.wl.x, lB, fmaf(k.wr.x, c.B[ch].y, sB.x));
        sB.y = fmaf(k.wl.y, c.B[ch].x, fmaf(k.wr.y, rB, sB.y));
        const float2 bF = fma2(k.a, k.I[ch], sF);              // alpha I + sum s_j F_j
        const float2 bB = fma2(be, k.I[ch], sB);               // (1-alpha) I + sum s_j B_j
        const float2 tF = mul2(k.nFB, bB);
        const float2 tB = mul2(k.nFB, bF);
        if (CLAMP) {
            out.F[ch] = f2(__saturatef(fmaf(k.mFF.x, bF.x, tF.x)), __saturatef(fmaf(k.mFF.y, bF.y, tF.y)));
            out.B[ch] = f2(__saturatef(fmaf(k.mBB.x, bB.x, tB.x)), __saturatef(fmaf(k.mBB.y, bB.y, tB.y)));
        } else {
            out.F[ch] = fma2(k.mFF, bF, tF);
            out.B[ch] = fma2(k.mBB, bB, tB);
        }
    }
}

// Output pointers of a lane: the bytes of its first pixel in row 0 of F and B.
struct Out {
    unsigned char *F, *B;
    long long pitch;        // bytes
    bool o0, o1;            // this lane writes p0 / p1
    const unsigned char *Bn;   // compositing epilogue (In == nullptr: none), same columns
    unsigned char *In;
    long long bn_pitch, in_pitch;   // bytes
};

// Two adjacent 16-bit elements in one 4-byte store (each rounded to nearest even).
__device__ __forceinline__ void st_pair(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void st_pair(__half *p, float a, float b) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void st_pair(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}

// Compositing epilogue of a lane's pixel pair in row r: In = alpha F + (1 - alpha) Bn.
template <typename T>
__device__ __forceinline__ void composite_row(const Out &o, int r, const FB &v, float2 a) {
    const T *Nr = reinterpret_cast<const T *>(o.Bn + (long long)r * o.bn_pitch);
    T *Cr = reinterpret_cast<T *>(o.In + (long long)r * o.in_pitch);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (o.o0) st_elem(Cr + c, fmaf(a.x, v.F[c].x, (1.f - a.x) * ld_elem(Nr + c)));
        if (o.o1) st_elem(Cr + 3 + c, fmaf(a.y, v.F[c].y, (1.f - a.y) * ld_elem(Nr + 3 + c)));
    }
}

template <typename T>
__device__ __forceinline__ void store_row(const Out &o, int r, const FB &v, float2 a) {
    if (o.In) composite_row<T>(o, r, v, a);
    T *Fr = reinterpret_cast<T *>(o.F + (long long)r * o.pitch);
    T *Br = reinterpret_cast<T *>(o.B + (long long)r * o.pitch);
    if (sizeof(T) == 4 && o.o0 && o.o1 &&
        (((uint32_t)reinterpret_cast<uintptr_t>(Fr) | (uint32_t)reinterpret_cast<uintptr_t>(Br)) & 7) == 0) {
        float2 *F2 = reinterpret_cast<float2 *>(Fr);
        float2 *B2 = reinterpret_cast<float2 *>(Br);
        F2[0] = f2(v.F[0].x, v.F[1].x);
        F2[1] = f2(v.F[2].x, v.F[0].y);
        F2[2] = f2(v.F[1].y, v.F[2].y);
        B2[0] = f2(v.B[0].x, v.B[1].x);
        B2[1] = f2(v.B[2].x, v.B[0].y);
        B2[2] = f2(v.B[1].y, v.B[2].y);
        return;
    }
    if (sizeof(T) == 2 && o.o0 && o.o1 &&
        (((uint32_t)reinterpret_cast<uintptr_t>(Fr) | (uint32_t)reinterpret_cast<uintptr_t>(Br)) & 3) == 0) {
        // six 16-bit values per image as three element pairs
        st_pair(Fr + 0, v.F[0].x, v.F[1].x);
        st_pair(Fr + 2, v.F[2].x, v.F[0].y);
        st_pair(Fr + 4, v.F[1].y, v.F[2].y);
        st_pair(Br + 0, v.B[0].x, v.B[1].x);
        st_pair(Br + 2, v.B[2].x, v.B[0].y);
        st_pair(Br + 4, v.B[1].y, v.B[2].y);
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (o.o0) {
            st_elem(Fr + c, v.F[c].x);
            st_elem(Br + c, v.B[c].x);
        }
        if (o.o1) {
            st_elem(Fr + 3 + c, v.F[c].y);
            st_elem(Br + 3 + c, v.B[c].y);
        }
    }
}

struct Ctl {
    int r_first, r_last;   // rows loaded
    int t1_lo, t1_hi;      // rows of sweep 1 (for K == 2)
    int Y0, Y1;            // output rows [Y0, Y1)
};

// ------------------------------------------------------------------ row sources

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// Loads of F and B written earlier in the same launch bypass the per-SM caches;
// everything else goes through the read-only path.
template <typename T, bool COHERENT>
__device__ __forceinline__ float ld_state(const T *p) {
    if (COHERENT) return to_f(__ldcg(p));
    return ld_elem(p);
}

// Register variant: plain loads of row r+1 issued while row r is processed.
template <typename T, bool COHERENT = false>
struct RegSource {
    Raw nxt;

    __device__ __forceinline__ void load(const PassArgs &p, const LaneGeo &g, int r, Raw &o) {
        const int gy = nearest_src(r, p.Ih, p.h);
        const int sy = nearest_src(r, p.sh, p.h);
        const T *Ir = static_cast<const T *>(p.I) + (long long)gy * p.I_pitch;
        const T *Ar = static_cast<const T *>(p.A) + (long long)gy * p.A_pitch;
        const T *Fr = static_cast<const T *>(p.Fs) + (long long)sy * p.s_pitch;
        const T *Br = static_cast<const T *>(p.Bs) + (long long)sy * p.s_pitch;
        o.a0 = ld_elem(Ar + g.gi0);
        o.a1 = ld_elem(Ar + g.gi1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.i0[c] = ld_elem(Ir + 3 * g.gi0 + c);
            o.i1[c] = ld_elem(Ir + 3 * g.gi1 + c);
            o.f0[c] = ld_state<T, COHERENT>(Fr + 3 * g.gs0 + c);
            o.f1[c] = ld_state<T, COHERENT>(Fr + 3 * g.gs1 + c);
            o.b0[c] = ld_state<T, COHERENT>(Br + 3 * g.gs0 + c);
            o.b1[c] = ld_state<T, COHERENT>(Br + 3 * g.gs1 + c);
        }
    }
    __device__ __forceinline__ void start(const PassArgs &p, const LaneGeo &g, const Ctl &ct) {
        load(p, g, ct.r_first, nxt);
    }
    __device__ __forceinline__ bool get(const PassArgs &p, const LaneGeo &g, const Ctl &ct, int r,
                                        Raw &out) {
        out = nxt;
        if (r + 1 <= ct.r_last) load(p, g, r + 1, nxt);
        return true;
    }
    __device__ __forceinline__ void abort() {}
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}


// floor((2r + 1) S / (2D)) for r = r0, r0 + 1, ... without a division per row.
struct RowMap {
    int q, rem, dq, drem, den;
    __device__ __forceinline__ void init(int r0, int S, int D) {
        const unsigned num = (2u * (unsigned)r0 + 1u) * (unsigned)S;
        den = 2 * D;
        q = (int)(num / (unsigned)den);
        rem = (int)(num % (unsigned)den);
        dq = (2 * S) / den;
        drem = (2 * S) % den;
    }
    __device__ __forceinline__ int next() {
        const int v = q;
        q += dq;
        rem += drem;
        if (rem >= den) {
            rem -= den;
            ++q;
        }
        return v;
    }
};

// Ring variant: the warp's rows r .. r + kRingSlots - 1 are in flight or resident in
// shared memory. A slot holds the four source segments of a row (I, alpha, F, B), each
// at a 16-byte aligned offset and copied by one bulk copy as the 16-byte aligned
// superset of its byte range. A segment whose superset could leave its image (only
// possible in the first or last row of that image) is checked, and copied by the
// lanes instead when it would.
template <typename T>
struct RingSource {
    uint32_t slots_s;       // shared address of this warp's first slot
    uint32_t bar0;          // shared address of this warp's first mbarrier
    int lane;
    int colI, colA, colS;   // byte offset of the strip's first source column in a row
    int lenI, lenA, lenS;   // bytes of each segment
    int li, la, ls, dI, dS; // per-lane element offsets inside the segments
    int fslot, gslot;       // next slot to fill / to take
    uint32_t fpar, gpar;    // their phase parities
    uint32_t issued;        // bit s: slot s has a fill in flight
    uint32_t parity;        // bit s: phase parity of slot s's fill in flight
    RowMap fI, fS, gI, gS;  // source rows of the next row to fill / to take

    __device__ __forceinline__ const unsigned char *row_addr(const PassArgs &p, int k, int y) const {
        const int es = (int)sizeof(T);
        switch (k) {
            case 0: return static_cast<const unsigned char *>(p.I) + (long long)y * p.I_pitch * es + colI;
            case 1: return static_cast<const unsigned char *>(p.A) + (long long)y * p.A_pitch * es + colA;
            case 2: return static_cast<const unsigned char *>(p.Fs) + (long long)y * p.s_pitch * es + colS;
            default: return static_cast<const unsigned char *>(p.Bs) + (long long)y * p.s_pitch * es + colS;
        }
    }
    __device__ __forceinline__ int seg_len(int k) const {
        return k == 0 ? lenI : k == 1 ? lenA : lenS;
    }
    __device__ __forceinline__ uint32_t seg_off(const PassArgs &p, int k) const {
        return k == 0 ? 0u : k == 1 ? (uint32_t)p.capI
                                    : k == 2 ? (uint32_t)(p.capI + p.capA)
                                             : (uint32_t)(p.capI + p.capA + p.capS);
    }

    // Warp-collective: start filling slot fslot with the next row.
    __device__ __forceinline__ void fill(const PassArgs &p) {
        const int gy = fI.next(), sy = fS.next();
        const uint32_t slot_s = slots_s + (uint32_t)fslot * (uint32_t)p.slot_bytes;
        const uint32_t bar = bar0 + 8u * (uint32_t)fslot;
        const bool edgeI = gy == 0 || gy == p.Ih - 1;
        const bool edgeS = sy == 0 || sy == p.sh - 1;
        uint32_t tx = 0;
        bool bulk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned char *a = row_addr(p, k, k < 2 ? gy : sy);
            const uintptr_t a16 = reinterpret_cast<uintptr_t>(a) & ~(uintptr_t)15;
            const uint32_t n = ((((uint32_t)reinterpret_cast<uintptr_t>(a) & 15u) + (uint32_t)seg_len(k) + 15u) & ~15u);
            bulk[k] = true;
            if (k < 2 ? edgeI : edgeS) {
                const void *lo = k == 0 ? p.I : k == 1 ? p.A : k == 2 ? p.Fs : p.Bs;
                const void *hi = k == 0 ? p.I_end : k == 1 ? p.A_end : k == 2 ? p.Fs_end : p.Bs_end;
                bulk[k] = a16 >= reinterpret_cast<uintptr_t>(lo) &&
                          a16 + n <= reinterpret_cast<uintptr_t>(hi);
            }
            if (bulk[k]) {
                tx += n;
            } else {
                // the aligned superset would leave the image: copy the elements by lanes
                const uint32_t dst = slot_s + seg_off(p, k) + ((uint32_t)reinterpret_cast<uintptr_t>(a) & 15u);
                const T *src = reinterpret_cast<const T *>(a);
                for (int e = lane; e < seg_len(k) / (int)sizeof(T); e += 32) {
                    T v = __ldcg(src + e);
                    unsigned short u;
                    if (sizeof(T) == 4) {
                        asm volatile("st.shared.b32 [%0], %1;" :: "r"(dst + 4u * e), "r"(__float_as_uint(*reinterpret_cast<float *>(&v))) : "memory");
                    } else {
                        u = *reinterpret_cast<unsigned short *>(&v);
                        asm volatile("st.shared.b16 [%0], %1;" :: "r"(dst + 2u * e), "h"(u) : "memory");
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(bar), "r"(tx) : "memory");
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!bulk[k]) continue;
                const unsigned char *a = row_addr(p, k, k < 2 ? gy : sy);
                const uintptr_t a16 = reinterpret_cast<uintptr_t>(a) & ~(uintptr_t)15;
                const uint32_t n = ((((uint32_t)reinterpret_cast<uintptr_t>(a) & 15u) + (uint32_t)seg_len(k) + 15u) & ~15u);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    :: "r"(slot_s + seg_off(p, k)), "l"(a16), "r"(n), "r"(bar)
                    : "memory");
            }
        }
        issued |= 1u << fslot;
        parity = (parity & ~(1u << fslot)) | (fpar << fslot);
        if (++fslot == kRingSlots) {
            fslot = 0;
            fpar ^= 1u;
        }
    }

    // Bounded wait for phase `par` of `slot`; warp-uniform result.
    __device__ __forceinline__ bool wait(int slot, uint32_t par) const {
        const uint32_t bar = bar0 + 8u * (uint32_t)slot;
        uint32_t ok = 0;
        for (int i = 0; i < kWaitPolls && !ok; ++i) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok) : "r"(bar), "r"(par), "r"(kWaitHintNs) : "memory");
        }
        return __all_sync(kFull, ok != 0);
    }

    // The strip's source column ranges: lanes load columns [xf, xl] of the level.
    __device__ __forceinline__ void setup(const PassArgs &p, const LaneGeo &g, int ln) {
        const int X0 = g.x - 2 * ln;
        const int xf = min(max(X0, 0), p.w - 1);
        const int xl = min(max(X0 + kLaneCols - 1, 0), p.w - 1);
        const int giF = nearest_src(xf, p.Iw, p.w);
        const int nI = nearest_src(xl, p.Iw, p.w) - giF + 1;
        const int gsF = nearest_src(xf, p.sw, p.w);
        const int nS = nearest_src(xl, p.sw, p.w) - gsF + 1;
        const int es = (int)sizeof(T);
        colI = 3 * giF * es;
        colA = giF * es;
        colS = 3 * gsF * es;
        lenI = 3 * nI * es;
        lenA = nI * es;
        lenS = 3 * nS * es;
        li = 3 * (g.gi0 - giF);
        la = g.gi0 - giF;
        ls = 3 * (g.gs0 - gsF);
        dI = g.gi1 - g.gi0;
        dS = g.gs1 - g.gs0;
    }

    __device__ __forceinline__ void start(const PassArgs &p, const LaneGeo &g, const Ctl &ct) {
        fI.init(ct.r_first, p.Ih, p.h);
        fS.init(ct.r_first, p.sh, p.h);
        gI.init(ct.r_first, p.Ih, p.h);
        gS.init(ct.r_first, p.sh, p.h);
        for (int i = 0; i < kRingSlots && ct.r_first + i <= ct.r_last; ++i) fill(p);
    }

    __device__ __forceinline__ bool get(const PassArgs &p, const LaneGeo &g, const Ctl &ct, int r,
                                        Raw &o) {
        const int slot = gslot;
        if (!wait(slot, gpar)) return false;
        issued &= ~(1u << slot);
        if (++gslot == kRingSlots) {
            gslot = 0;
            gpar ^= 1u;
        }
        const int gy = gI.next(), sy = gS.next();
        const uint32_t slot_s = slots_s + (uint32_t)slot * (uint32_t)p.slot_bytes;
        // slack of each segment inside its 16-byte aligned superset
        const uint32_t sI = (uint32_t)reinterpret_cast<uintptr_t>(row_addr(p, 0, gy)) & 15u;
        const uint32_t sA = (uint32_t)reinterpret_cast<uintptr_t>(row_addr(p, 1, gy)) & 15u;
        const uint32_t sF = (uint32_t)reinterpret_cast<uintptr_t>(row_addr(p, 2, sy)) & 15u;
        const uint32_t sB = (uint32_t)reinterpret_cast<uintptr_t>(row_addr(p, 3, sy)) & 15u;
        const int es = (int)sizeof(T);
        const uint32_t I = slot_s + sI + (uint32_t)(li * es);
        const uint32_t A = slot_s + (uint32_t)p.capI + sA + (uint32_t)(la * es);
        const uint32_t F = slot_s + (uint32_t)(p.capI + p.capA) + sF + (uint32_t)(ls * es);
        const uint32_t B = slot_s + (uint32_t)(p.capI + p.capA + p.capS) + sB + (uint32_t)(ls * es);
        o.a0 = lds<T>(A);
        o.a1 = lds<T>(A + dI * es);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.i0[c] = lds<T>(I + c * es);
            o.i1[c] = lds<T>(I + (3 * dI + c) * es);
            o.f0[c] = lds<T>(F + c * es);
            o.f1[c] = lds<T>(F + (3 * dS + c) * es);
            o.b0[c] = lds<T>(B + c * es);
            o.b1[c] = lds<T>(B + (3 * dS + c) * es);
        }
        __syncwarp();   // every lane has read the slot before it is refilled
        if (r + kRingSlots <= ct.r_last) fill(p);
        return true;
    }

    const unsigned char *sm;   // the block's shared memory, and its shared address
    uint32_t sbase;
    template <typename U>
    __device__ __forceinline__ float lds(uint32_t a) const {
        return to_f(*reinterpret_cast<const U *>(sm + (a - sbase)));
    }

    // After a failed wait: wait (bounded) for every fill still in flight, then return.
    __device__ __forceinline__ void abort() const {
        for (int s = 0; s < kRingSlots; ++s)
            if (issued & (1u << s)) wait(s, (parity >> s) & 1u);
    }
};

// ------------------------------------------------------------------ the pass

// One row step: take row r, finish the weights of row r-1, sweep 1 at row r-1 and
// (K == 2) sweep 2 at row r-2. Queue arguments are the rows r, r-1, r-2 (S: row data,
// Q: starting state) and r-1, r-2, r-3 (P: sweep-1 state). Returns false if a bounded
// wait gave up.
//
// STEADY: every stage is active and no image border is involved (the caller checks the
// row range), so the step runs without guards and its stages form one basic block that
// the compiler can interleave.
template <typename T, int K, bool CLAMP, bool STEADY, typename Src>
__device__ __forceinline__ bool step(const PassArgs &p, const LaneGeo &g, const Ctl &ct,
                                     const Out &out, int r, Src &src, RowK &Sr, RowK &Sr1,
                                     RowK &Sr2, FB &Qr, FB &Qr1, FB &Qr2, FB &Pw, FB &Pr2,
                                     FB &Pr3) {
    if (STEADY || r <= ct.r_last) {
        Raw cur;
        if (!src.get(p, g, ct, r, cur)) return false;
        make_row(cur, g, STEADY ? 1 : r, Sr1, p.eps, p.omega, Sr, Qr);
    }
    const int q = r - 1;
    if (STEADY || (q >= ct.r_first && q <= ct.r_last)) {
        if (STEADY || q < p.h - 1) {
            Sr1.wd = Sr.wu;          // the edge (q, q+1) seen from row q
        } else {
            Sr1.wd = f2(0.f, 0.f);   // bottom row: the neighbour below is the pixel itself
            Sr1.ws = add2(Sr1.ws, f2(p.eps, p.eps));
        }
        finish_row(Sr1);
    }
    if (K == 1) {
        if (STEADY || (q >= ct.Y0 && q < ct.Y1)) {
            FB res;
            update<CLAMP>(Sr1, Qr1, Qr2, Qr, res);
            store_row<T>(out, q, res, Sr1.a);
        }
    } else {
        if (STEADY || (q >= ct.t1_lo && q <= ct.t1_hi)) update<CLAMP>(Sr1, Qr1, Qr2, Qr, Pw);
        const int q2 = r - 2;
        if (STEADY || (q2 >= ct.Y0 && q2 < ct.Y1)) {
            FB res;
            update<CLAMP>(Sr2, Pr2, Pr3, Pw, res);
            store_row<T>(out, q2, res, Sr2.a);
        }
    }
    return true;
}

// Rows r whose step has every stage active and touches no image border.
__device__ __forceinline__ void steady_range(const Ctl &ct, int K, int &lo, int &hi) {
    if (K == 1) {
        lo = max(max(ct.r_first + 1, ct.Y0 + 1), 1);
        hi = min(ct.r_last, ct.Y1);
    } else {
        lo = max(max(ct.r_first + 2, ct.t1_lo + 1), max(ct.Y0 + 2, 1));
        hi = min(ct.r_last, min(ct.t1_hi + 1, ct.Y1 + 1));
    }
}

__device__ __forceinline__ void zero(FB &v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v.F[c] = v.B[c] = f2(0.f, 0.f);
}
__device__ __forceinline__ void zero(RowK &v) {
    v.a = v.wl = v.wr = v.wu = v.wd = v.ws = v.mFF = v.mBB = v.nFB = f2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) v.I[c] = f2(0.f, 0.f);
}

template <typename T>
__device__ __forceinline__ void lane_setup(const PassArgs &p, int warp, int lane, LaneGeo &g,
                                           Ctl &ct, Out &out, int K) {
    const int xs = warp % p.n_xstrips;
    const int ys = warp / p.n_xstrips;
    g.x = xs * kStripW - 2 + 2 * lane;
    const int xc0 = min(max(g.x, 0), p.w - 1);
    const int xc1 = min(max(g.x + 1, 0), p.w - 1);
    g.gi0 = nearest_src(xc0, p.Iw, p.w);
    g.gi1 = nearest_src(xc1, p.Iw, p.w);
    g.gs0 = nearest_src(xc0, p.sw, p.w);
    g.gs1 = nearest_src(xc1, p.sw, p.w);
    g.inL0 = g.x > 0;
    g.inR0 = g.x + 1 < p.w;
    g.inR1 = g.x + 2 < p.w;
    ct.Y0 = ys * p.strip_h;
    ct.Y1 = min(ct.Y0 + p.strip_h, p.h);
    ct.r_first = max(ct.Y0 - K, 0);
    ct.r_last = min(ct.Y1 - 1 + K, p.h - 1);
    ct.t1_lo = max(ct.Y0 - 1, 0);
    ct.t1_hi = min(ct.Y1, p.h - 1);
    const bool mid = lane >= 1 && lane <= 30;
    out.o0 = mid && g.x < p.w;
    out.o1 = mid && g.x + 1 < p.w;
    const long long col = 3LL * max(g.x, 0) * (long long)sizeof(T);
    out.F = static_cast<unsigned char *>(p.Fd) + col;
    out.B = static_cast<unsigned char *>(p.Bd) + col;
    out.pitch = p.d_pitch * (long long)sizeof(T);
    out.In = p.In ? static_cast<unsigned char *>(p.In) + col : nullptr;
    out.Bn = p.In ? static_cast<const unsigned char *>(p.Bn) + col : nullptr;
    out.bn_pitch = p.bn_pitch * (long long)sizeof(T);
    out.in_pitch = p.in_pitch * (long long)sizeof(T);
}

template <typename T, int K, bool CLAMP, typename Src>
__device__ __forceinline__ bool run_strip(const PassArgs &p, const LaneGeo &g, const Ctl &ct,
                                          const Out &out, Src &src) {
    RowK S0, S1, S2;
    FB Q0, Q1, Q2, P0, P1, P2;
    zero(S0); zero(S1); zero(S2);
    zero(Q0); zero(Q1); zero(Q2);
    zero(P0); zero(P1); zero(P2);
    src.start(p, g, ct);
    const int r_end = ct.r_last + K;
    int s_lo, s_hi;
    steady_range(ct, K, s_lo, s_hi);
    bool ok = true;
#define FGML_STEP(R, A, B, C, D, E, F, G, H, I)                                                      \
    ((R) >= s_lo && (R) <= s_hi                                                                      \
         ? step<T, K, CLAMP, true>(p, g, ct, out, (R), src, A, B, C, D, E, F, G, H, I)               \
         : step<T, K, CLAMP, false>(p, g, ct, out, (R), src, A, B, C, D, E, F, G, H, I))
    for (int r = ct.r_first; r <= r_end && ok; r += 3) {
        ok = FGML_STEP(r, S0, S2, S1, Q0, Q2, Q1, P2, P1, P0);
        if (!ok || r + 1 > r_end) break;
        ok = FGML_STEP(r + 1, S1, S0, S2, Q1, Q0, Q2, P0, P2, P1);
        if (!ok || r + 2 > r_end) break;
        ok = FGML_STEP(r + 2, S2, S1, S0, Q2, Q1, Q0, P1, P0, P2);
    }
#undef FGML_STEP
    if (!ok) {
        if ((threadIdx.x & 31) == 0) atomicExch(&g_device_error, 1);
        src.abort();
    }
    return ok;
}

template <typename T, int K, bool CLAMP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) level_pass_kernel(const PassArgs p) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (warp >= p.n_warps) return;
    LaneGeo g;
    Ctl ct;
    Out out;
    lane_setup<T>(p, warp, lane, g, ct, out, K);
    RegSource<T> src;
    run_strip<T, K, CLAMP>(p, g, ct, out, src);
    pdl_leave();
}

template <typename T, int K, bool CLAMP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kRingMinBlocks) level_pass_ring_kernel(const PassArgs p) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (warp >= p.n_warps) return;
    LaneGeo g;
    Ctl ct;
    Out out;
    lane_setup<T>(p, warp, lane, g, ct, out, K);

    RingSource<T> src;
    src.sm = smem;
    src.sbase = smem_addr(smem);
    src.lane = lane;
    src.slots_s = smem_addr(smem) + (uint32_t)(wib * kRingSlots * p.slot_bytes);
    src.bar0 = smem_addr(smem) + (uint32_t)(kWarpsPerBlock * kRingSlots * p.slot_bytes) +
               8u * (uint32_t)(wib * kRingSlots);
    src.fslot = src.gslot = 0;
    src.fpar = src.gpar = 0;
    src.issued = src.parity = 0;
    src.setup(p, g, lane);
    if (lane == 0) {
        for (int s = 0; s < kRingSlots; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(src.bar0 + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    run_strip<T, K, CLAMP>(p, g, ct, out, src);
    pdl_leave();
}

// Zero sweeps: the level's F and B are the nearest resize of the starting state.
template <typename T>
__global__ void resize_fb_kernel(const PassArgs p) {
    pdl_enter();
    const long long n = (long long)p.w * p.h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.w), y = (int)(i / p.w);
        const int sx = nearest_src(x, p.sw, p.w), sy = nearest_src(y, p.sh, p.h);
        const T *Fs = static_cast<const T *>(p.Fs) + (long long)sy * p.s_pitch + 3 * sx;
        const T *Bs = static_cast<const T *>(p.Bs) + (long long)sy * p.s_pitch + 3 * sx;
        T *Fd = static_cast<T *>(p.Fd) + (long long)y * p.d_pitch + 3 * x;
        T *Bd = static_cast<T *>(p.Bd) + (long long)y * p.d_pitch + 3 * x;
        for (int c = 0; c < 3; ++c) {
            Fd[c] = Fs[c];
            Bd[c] = Bs[c];
        }
        if (p.In) {
            const float F[3] = {to_f(Fs[0]), to_f(Fs[1]), to_f(Fs[2])};
            const int gx = nearest_src(x, p.Iw, p.w), gy = nearest_src(y, p.Ih, p.h);
            const float a = ld_elem(static_cast<const T *>(p.A) + (long long)gy * p.A_pitch + gx);
            composite_px<T>(p.Bn, p.bn_pitch, p.In, p.in_pitch, x, y, a, F);
        }
    }
    pdl_leave();
}

template <typename T, int K, bool CLAMP>
cudaError_t launch_t(const PassArgs &a, cudaStream_t s) {
    const int blocks = (a.n_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return launch_pdl(level_pass_kernel<T, K, CLAMP>, dim3(blocks), dim3(kWarpsPerBlock * 32), 0, s, a);
}

template <typename T, int K, bool CLAMP>
cudaError_t launch_ring_t(const PassArgs &a, cudaStream_t s) {
    const int blocks = (a.n_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const size_t smem = level_pass_ring_smem(a.slot_bytes);
    cudaError_t e = allow_dynamic_smem(level_pass_ring_kernel<T, K, CLAMP>);
    if (e != cudaSuccess) return e;
    return launch_pdl(level_pass_ring_kernel<T, K, CLAMP>, dim3(blocks), dim3(kWarpsPerBlock * 32), smem, s, a);
}

template <typename T>
cudaError_t launch_dtype(int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if (iters == 0) {
        const long long n = (long long)a.w * a.h;
        const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
        return launch_pdl(resize_fb_kernel<T>, dim3(blocks), dim3(256), 0, s, a);
    }
    if (iters == 1) return clamp ? launch_t<T, 1, true>(a, s) : launch_t<T, 1, false>(a, s);
    return clamp ? launch_t<T, 2, true>(a, s) : launch_t<T, 2, false>(a, s);
}

template <typename T>
cudaError_t launch_ring_dtype(int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if (iters == 1) return clamp ? launch_ring_t<T, 1, true>(a, s) : launch_ring_t<T, 1, false>(a, s);
    if (iters == 2) return clamp ? launch_ring_t<T, 2, true>(a, s) : launch_ring_t<T, 2, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_level_pass(int dtype, int iters, int clamp, const PassArgs &a,
                              cudaStream_t s) {
    if (iters < 0 || iters > 2) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return launch_dtype<float>(iters, clamp, a, s);
        case kBF16: return launch_dtype<__nv_bfloat16>(iters, clamp, a, s);
        case kF16: return launch_dtype<__half>(iters, clamp, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_level_pass_ring(int dtype, int iters, int clamp, const PassArgs &a,
                                   cudaStream_t s) {
    if (a.slot_bytes <= 0 || (a.slot_bytes & 15) || (a.capI & 15) || (a.capA & 15) ||
        (a.capS & 15))
        return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return launch_ring_dtype<float>(iters, clamp, a, s);
        case kBF16: return launch_ring_dtype<__nv_bfloat16>(iters, clamp, a, s);
        case kF16: return launch_ring_dtype<__half>(iters, clamp, a, s);
    }
    return cudaErrorInvalidValue;
}

int level_pass_tile_rows() { return kTileRows; }

size_t level_pass_ring_smem(int slot_bytes) {
    return (size_t)kWarpsPerBlock * kRingSlots * (size_t)slot_bytes +
           (size_t)kWarpsPerBlock * kRingSlots * 8;
}

int strip_span(int S, int D) {
    int best = 1;
    const int nx = (D + kStripW - 1) / kStripW;
    for (int xs = 0; xs < nx; ++xs) {
        const int X0 = xs * kStripW - 2;
        const int xf = std::min(std::max(X0, 0), D - 1);
        const int xl = std::min(std::max(X0 + kLaneCols - 1, 0), D - 1);
        best = std::max(best, nearest_src(xl, S, D) - nearest_src(xf, S, D) + 1);
    }
    return best;
}

cudaError_t read_and_clear_device_error(int *code, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(code, g_device_error, sizeof(int), 0,
                                              cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*code) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_device_error, &zero, sizeof(int), 0,
                                    cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
    }
    int tile = 0;   // the tile kernel's own error word (level_tile.cu)
    e = read_and_clear_tile_error(&tile, s);
    if (e == cudaSuccess && !*code) *code = tile;
    return e;
}

cudaError_t enqueue_device_error_read(int *dst, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(dst, g_device_error, sizeof(int), 0,
                                              cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? enqueue_tile_error_read(dst + 1, s) : e;
}

int level_pass_strip_width() { return kStripW; }
int level_pass_warps_per_block() { return kWarpsPerBlock; }

}  // namespace fgml
