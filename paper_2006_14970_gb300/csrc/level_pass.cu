// Level pass: K Jacobi sweeps of one pyramid level in a single trip through HBM.
//
// Each warp owns a strip of 64 columns (two adjacent pixels per lane) and walks down
// its rows. Row r of the starting state is gathered from HBM exactly once (alpha and I
// by nearest resize of the full-resolution input, F and B by nearest resize of the
// previous level, Algorithm 1), sweep 1 is computed one row behind the loads and sweep 2
// one row behind sweep 1, all in registers: three-row register queues per sweep, left
// and right neighbours through warp shuffles. The two outermost columns of the strip
// are halo, so a warp writes 60 columns; the strip's vertical halo is K rows.
//
// The per-pixel update is the closed-form 2x2 solve of Section III-C,
//   g = (U U^T + S I_2)^{-1} (U I + sum_j s_j [F_j; B_j]),  U = (alpha, 1 - alpha),
// with s_j = eps_r + omega |alpha_i - alpha_j| over the 4-neighbourhood and S = sum s_j,
// solved through the adjugate and clamped to [0, 1] (Algorithm 1). A neighbour outside
// the image is the pixel itself (Algorithm 1 clamps coordinates): its weight is eps_r
// and its value the pixel's own previous value. Pairs of pixels use the packed
// float32x2 arithmetic of sm_100-class GPUs.
#include "fgml_internal.h"

#include <algorithm>

namespace fgml {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 60;          // output columns per warp
constexpr int kWarpsPerBlock = 4;

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
};

struct Raw {                // one row as loaded
    float a0, a1;
    float i0[3], i1[3];
    float f0[3], f1[3], b0[3], b1[3];
};

struct LaneGeo {
    int x;                  // column of the lane's first pixel (may be outside the image)
    int oi0, oi1;           // element offsets of the two pixels in a row of I
    int oa0, oa1;           // ... in a row of alpha
    int os0, os1;           // ... in a row of the starting F and B
    bool inL0, inR0, inR1;  // left of p0, right of p0, right of p1 lie inside the image
};

template <typename T>
__device__ __forceinline__ void load_raw(const PassArgs &p, const LaneGeo &g, int r, Raw &o) {
    const int gy = nearest_src(r, p.Ih, p.h);
    const int sy = nearest_src(r, p.sh, p.h);
    const T *Ir = static_cast<const T *>(p.I) + (long long)gy * p.I_pitch;
    const T *Ar = static_cast<const T *>(p.A) + (long long)gy * p.A_pitch;
    const T *Fr = static_cast<const T *>(p.Fs) + (long long)sy * p.s_pitch;
    const T *Br = static_cast<const T *>(p.Bs) + (long long)sy * p.s_pitch;
    o.a0 = ld_elem(Ar + g.oa0);
    o.a1 = ld_elem(Ar + g.oa1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.i0[c] = ld_elem(Ir + g.oi0 + c);
        o.i1[c] = ld_elem(Ir + g.oi1 + c);
        o.f0[c] = ld_elem(Fr + g.os0 + c);
        o.f1[c] = ld_elem(Fr + g.os1 + c);
        o.b0[c] = ld_elem(Br + g.os0 + c);
        o.b1[c] = ld_elem(Br + g.os1 + c);
    }
}

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

// One Jacobi update of a row: c = the row's previous state, up/dn = the previous state
// of the rows above and below (ignored where the weight is 0).
template <bool CLAMP>
__device__ __forceinline__ void update(const RowK &k, const FB &c, const FB &up, const FB &dn,
                                       FB &out) {
    const float2 S = add2(add2(add2(k.wl, k.wr), add2(k.wu, k.wd)), k.ws);
    const float2 be = f2(1.f - k.a.x, 1.f - k.a.y);           // 1 - alpha
    const float2 A00 = fma2(k.a, k.a, S);                      // alpha^2 + S
    const float2 A11 = fma2(be, be, S);                        // (1 - alpha)^2 + S
    const float2 A01 = mul2(k.a, be);                          // alpha (1 - alpha)
    const float2 det = fma2(A00, A11, neg2(mul2(A01, A01)));
    const float2 m = f2(__frcp_rn(det.x), __frcp_rn(det.y));
    const float2 mFF = mul2(A11, m), mBB = mul2(A00, m), nFB = neg2(mul2(A01, m));
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float lF = __shfl_up_sync(kFull, c.F[ch].y, 1);
        const float rF = __shfl_down_sync(kFull, c.F[ch].x, 1);
        const float lB = __shfl_up_sync(kFull, c.B[ch].y, 1);
        const float rB = __shfl_down_sync(kFull, c.B[ch].x, 1);
        float2 sF = mul2(k.ws, c.F[ch]);
        sF = fma2(k.wl, f2(lF, c.F[ch].x), sF);
        sF = fma2(k.wr, f2(c.F[ch].y, rF), sF);
        sF = fma2(k.wu, up.F[ch], sF);
        sF = fma2(k.wd, dn.F[ch], sF);
        float2 sB = mul2(k.ws, c.B[ch]);
        sB = fma2(k.wl, f2(lB, c.B[ch].x), sB);
        sB = fma2(k.wr, f2(c.B[ch].y, rB), sB);
        sB = fma2(k.wu, up.B[ch], sB);
        sB = fma2(k.wd, dn.B[ch], sB);
        const float2 bF = fma2(k.a, k.I[ch], sF);              // alpha I + sum s_j F_j
        const float2 bB = fma2(be, k.I[ch], sB);               // (1-alpha) I + sum s_j B_j
        const float2 tF = mul2(nFB, bB);
        const float2 tB = mul2(nFB, bF);
        if (CLAMP) {
            out.F[ch] = f2(__saturatef(fmaf(mFF.x, bF.x, tF.x)), __saturatef(fmaf(mFF.y, bF.y, tF.y)));
            out.B[ch] = f2(__saturatef(fmaf(mBB.x, bB.x, tB.x)), __saturatef(fmaf(mBB.y, bB.y, tB.y)));
        } else {
            out.F[ch] = fma2(mFF, bF, tF);
            out.B[ch] = fma2(mBB, bB, tB);
        }
    }
}

template <typename T>
__device__ __forceinline__ void store_row(const PassArgs &p, const LaneGeo &g, int r,
                                          const FB &v, bool o0, bool o1) {
    T *Fr = static_cast<T *>(p.Fd) + (long long)r * p.d_pitch + 3 * g.x;
    T *Br = static_cast<T *>(p.Bd) + (long long)r * p.d_pitch + 3 * g.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (o0) {
            st_elem(Fr + c, v.F[c].x);
            st_elem(Br + c, v.B[c].x);
        }
        if (o1) {
            st_elem(Fr + 3 + c, v.F[c].y);
            st_elem(Br + 3 + c, v.B[c].y);
        }
    }
}

struct Ctl {
    int r_first, r_last;   // rows loaded
    int t1_lo, t1_hi;      // rows of sweep 1 (for K == 2)
    int Y0, Y1;            // output rows [Y0, Y1)
    bool o0, o1;           // this lane writes p0 / p1
};

// One row step: load row r, finish the weights of row r-1, sweep 1 at row r-1 and
// (K == 2) sweep 2 at row r-2. Queue arguments are the rows r, r-1, r-2 (S: row data,
// Q: starting state) and r-1, r-2, r-3 (P: sweep-1 state).
template <typename T, int K, bool CLAMP>
__device__ __forceinline__ void step(const PassArgs &p, const LaneGeo &g, const Ctl &ct, int r,
                                     Raw &nxt, RowK &Sr, RowK &Sr1, RowK &Sr2,
                                     FB &Qr, FB &Qr1, FB &Qr2, FB &Pw, FB &Pr2, FB &Pr3) {
    if (r <= ct.r_last) {
        const Raw cur = nxt;
        if (r + 1 <= ct.r_last) load_raw<T>(p, g, r + 1, nxt);
        make_row(cur, g, r, Sr1, p.eps, p.omega, Sr, Qr);
    }
    const int q = r - 1;
    if (q >= ct.r_first && q <= ct.r_last) {
        if (q < p.h - 1) {
            Sr1.wd = Sr.wu;          // the edge (q, q+1) seen from row q
        } else {
            Sr1.wd = f2(0.f, 0.f);   // bottom row: the neighbour below is the pixel itself
            Sr1.ws = add2(Sr1.ws, f2(p.eps, p.eps));
        }
    }
    if (K == 1) {
        if (q >= ct.Y0 && q < ct.Y1) {
            FB res;
            update<CLAMP>(Sr1, Qr1, Qr2, Qr, res);
            store_row<T>(p, g, q, res, ct.o0, ct.o1);
        }
    } else {
        if (q >= ct.t1_lo && q <= ct.t1_hi) update<CLAMP>(Sr1, Qr1, Qr2, Qr, Pw);
        const int q2 = r - 2;
        if (q2 >= ct.Y0 && q2 < ct.Y1) {
            FB res;
            update<CLAMP>(Sr2, Pr2, Pr3, Pw, res);
            store_row<T>(p, g, q2, res, ct.o0, ct.o1);
        }
    }
}

__device__ __forceinline__ void zero(FB &v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v.F[c] = v.B[c] = f2(0.f, 0.f);
}
__device__ __forceinline__ void zero(RowK &v) {
    v.a = v.wl = v.wr = v.wu = v.wd = v.ws = f2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) v.I[c] = f2(0.f, 0.f);
}

template <typename T, int K, bool CLAMP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) level_pass_kernel(const PassArgs p) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (warp >= p.n_warps) return;
    const int xs = warp % p.n_xstrips;
    const int ys = warp / p.n_xstrips;

    LaneGeo g;
    g.x = xs * kStripW - 2 + 2 * lane;
    const int xc0 = min(max(g.x, 0), p.w - 1);
    const int xc1 = min(max(g.x + 1, 0), p.w - 1);
    const int gi0 = nearest_src(xc0, p.Iw, p.w), gi1 = nearest_src(xc1, p.Iw, p.w);
    const int gs0 = nearest_src(xc0, p.sw, p.w), gs1 = nearest_src(xc1, p.sw, p.w);
    g.oi0 = 3 * gi0;
    g.oi1 = 3 * gi1;
    g.oa0 = gi0;
    g.oa1 = gi1;
    g.os0 = 3 * gs0;
    g.os1 = 3 * gs1;
    g.inL0 = g.x > 0;
    g.inR0 = g.x + 1 < p.w;
    g.inR1 = g.x + 2 < p.w;

    Ctl ct;
    ct.Y0 = ys * p.strip_h;
    ct.Y1 = min(ct.Y0 + p.strip_h, p.h);
    ct.r_first = max(ct.Y0 - K, 0);
    ct.r_last = min(ct.Y1 - 1 + K, p.h - 1);
    ct.t1_lo = max(ct.Y0 - 1, 0);
    ct.t1_hi = min(ct.Y1, p.h - 1);
    const bool mid = lane >= 1 && lane <= 30;
    ct.o0 = mid && g.x < p.w;
    ct.o1 = mid && g.x + 1 < p.w;

    RowK S0, S1, S2;
    FB Q0, Q1, Q2, P0, P1, P2;
    zero(S0); zero(S1); zero(S2);
    zero(Q0); zero(Q1); zero(Q2);
    zero(P0); zero(P1); zero(P2);
    Raw nxt;
    load_raw<T>(p, g, ct.r_first, nxt);

    const int r_end = ct.r_last + K;
    for (int r = ct.r_first; r <= r_end; r += 3) {
        step<T, K, CLAMP>(p, g, ct, r, nxt, S0, S2, S1, Q0, Q2, Q1, P2, P1, P0);
        if (r + 1 > r_end) break;
        step<T, K, CLAMP>(p, g, ct, r + 1, nxt, S1, S0, S2, Q1, Q0, Q2, P0, P2, P1);
        if (r + 2 > r_end) break;
        step<T, K, CLAMP>(p, g, ct, r + 2, nxt, S2, S1, S0, Q2, Q1, Q0, P1, P0, P2);
    }
}

// Zero sweeps: the level's F and B are the nearest resize of the starting state.
template <typename T>
__global__ void resize_fb_kernel(const PassArgs p) {
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
    }
}

template <typename T, int K, bool CLAMP>
cudaError_t launch_t(const PassArgs &a, cudaStream_t s) {
    const int blocks = (a.n_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    level_pass_kernel<T, K, CLAMP><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dtype(int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if (iters == 0) {
        const long long n = (long long)a.w * a.h;
        const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
        resize_fb_kernel<T><<<blocks, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (iters == 1) return clamp ? launch_t<T, 1, true>(a, s) : launch_t<T, 1, false>(a, s);
    return clamp ? launch_t<T, 2, true>(a, s) : launch_t<T, 2, false>(a, s);
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

int level_pass_strip_width() { return kStripW; }
int level_pass_warps_per_block() { return kWarpsPerBlock; }

}  // namespace fgml
