// Coarse levels: every level of at most 1024 pixels (with the paper's schedule, all
// the 10-sweep levels up to 32 x 32, Section III-D) runs inside one persistent
// 1024-thread block, from the 1x1 start of Algorithm 1 up to level `nlev`.
//  - I_l and alpha_l of every coarse level are gathered from the full-resolution input
//    (nearest resize, Algorithm 1). In float32 the gather is asynchronous (cp.async) in
//    two groups: the small levels' pixels, which the first sweeps wait for, and the rest,
//    which arrive while the small levels run.
//  - F and B live in shared memory as (F, B) pairs per channel, ping-ponged between two
//    buffers, with one barrier per Jacobi sweep over the warps that hold the level.
//  - Levels of at most 64 pixels run in three warps, one per channel, with each pixel's
//    (F, B) in registers and the neighbours taken by warp shuffles: a sweep is a short
//    dependent chain without shared memory or barriers. Larger levels run one thread per
//    pixel with (F, B) in shared memory.
//  - Each thread forms its pixel's neighbour weights and the inverse of its 2x2 matrix
//    (Section III-C) once per level; a sweep is then 4 neighbour reads, packed
//    multiply-adds and the clamped solve (Algorithm 1).
//  - With the red-black order an iteration is two in-place half-sweeps (x + y even, then
//    odd) over the one current buffer.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 1024;
constexpr int kSplitMax = 64;   // levels up to this many pixels run in registers, one warp per channel
constexpr unsigned kFull32 = 0xffffffffu;

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

template <typename T, bool CLAMP>
__device__ __forceinline__ void coarse_body(const CoarseArgs &p);

template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads, 1) coarse_kernel(const CoarseArgs p) {
    pdl_enter();
    // release the next launch at once: its blocks fetch their inputs while this single
    // block runs (they wait for this kernel before reading what it writes)
    pdl_leave();
    coarse_body<T, CLAMP>(p);
}

// One block per image of a batch; each reads its arguments from the device list.
template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads, 1) coarse_batch_kernel(const CoarseArgs *list) {
    coarse_body<T, CLAMP>(list[blockIdx.x]);
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Source pixel of gathered pixel `idx` (levels stored one after another from p.off[0]).
__device__ __forceinline__ void gather_src(const CoarseArgs &p, int idx, int &gx, int &gy) {
    int l = 0;
    while (l + 1 < p.nlev && p.off[l + 1] <= idx) ++l;
    const int w = p.lw[l], h = p.lh[l], i = idx - p.off[l];
    const int x = i % w, y = i / w;
    gx = nearest_src(x, p.Iw, w);
    gy = nearest_src(y, p.Ih, h);
}

// Barrier over the first nt threads (a multiple of 32) of the block.
__device__ __forceinline__ void level_sync(int nt) {
    if (nt == 32) __syncwarp();
    else if (nt == kThreads) __syncthreads();
    else asm volatile("bar.sync 1, %0;" :: "r"(nt) : "memory");
}

template <typename T, bool CLAMP>
__device__ __forceinline__ void coarse_body(const CoarseArgs &p) {
    extern __shared__ __align__(16) float sm[];
    // [0, 3 * kCoarseCap) float2: buffer X; then buffer Y; then per level I (3 floats per
    // pixel) and alpha, at the offsets p.off[l] (in pixels)
    float2 *const buf = reinterpret_cast<float2 *>(sm);
    float *Ilv = reinterpret_cast<float *>(buf + 2 * 3 * kCoarseCap);
    float *Alv = Ilv + 3 * p.total;
    const T *I = static_cast<const T *>(p.I);
    const T *A = static_cast<const T *>(p.A);
    const int tid = threadIdx.x;

    // pixels of the leading levels that run one thread per (pixel, channel)
    int split_px = 0;
    for (int l = 0; l < p.nlev && p.lw[l] * p.lh[l] <= kSplitMax; ++l) split_px = p.off[l] + p.lw[l] * p.lh[l];

    if (sizeof(T) == 4) {
        // asynchronous gather: group 0 the small levels, group 1 the rest
        const uint32_t sI = static_cast<uint32_t>(__cvta_generic_to_shared(Ilv));
        const uint32_t sA = static_cast<uint32_t>(__cvta_generic_to_shared(Alv));
        for (int g = 0; g < 2; ++g) {
            const int lo = g == 0 ? 0 : split_px, hi = g == 0 ? split_px : p.total;
            for (int idx = lo + tid; idx < hi; idx += kThreads) {
                int gx, gy;
                gather_src(p, idx, gx, gy);
                const T *Ip = I + (long long)gy * p.I_pitch + 3 * gx;
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_async4(sI + 4u * (3 * idx + c), Ip + c);
                cp_async4(sA + 4u * idx, A + (long long)gy * p.A_pitch + gx);
            }
            cp_async_commit();
        }
        cp_async_wait<1>();
    } else {
        // 16-bit storage: every load issued before any store
        constexpr int kPer = kCoarseTotal / kThreads;
        float gI[kPer][3], gA[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int idx = tid + k * kThreads;
            if (idx < p.total) {
                int gx, gy;
                gather_src(p, idx, gx, gy);
                const T *Ip = I + (long long)gy * p.I_pitch + 3 * gx;
                gI[k][0] = ld_elem(Ip + 0);
                gI[k][1] = ld_elem(Ip + 1);
                gI[k][2] = ld_elem(Ip + 2);
                gA[k] = ld_elem(A + (long long)gy * p.A_pitch + gx);
            }
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int idx = tid + k * kThreads;
            if (idx < p.total) {
                Ilv[3 * idx + 0] = gI[k][0];
                Ilv[3 * idx + 1] = gI[k][1];
                Ilv[3 * idx + 2] = gI[k][2];
                Alv[idx] = gA[k];
            }
        }
    }
    int cur = 0;   // buffer holding the current state: buf + cur * 3 * kCoarseCap
    if (tid == 0)
        for (int c = 0; c < 3; ++c) buf[c * kCoarseCap] = f2(p.init, p.init);   // 1 x 1 start

    int pw = 1, ph = 1;
    bool rest_waited = false;
    for (int l = 0; l < p.nlev; ++l) {
        const int w = p.lw[l], h = p.lh[l], k = p.lk[l], n = w * h, o = p.off[l];
        const bool split = n <= kSplitMax;
        if (!split && !rest_waited && sizeof(T) == 4) {
            cp_async_wait<0>();
            rest_waited = true;
        }
        __syncthreads();   // the previous level (and the gathered inputs) are visible
        if (split) {
            // up to 64 pixels: warp c holds channel c of every pixel in registers (pixels
            // lane and lane + 32) and takes its neighbours by shuffles; the channels are
            // independent given the weights, so no barrier is needed between sweeps
            if (tid < 3 * 32) {
                const int c = tid >> 5, lane = tid & 31;
                const float2 *src = buf + cur * 3 * kCoarseCap + c * kCoarseCap;
                float2 *dst = buf + (cur ^ 1) * 3 * kCoarseCap + c * kCoarseCap;
                const bool two = n > 32;
                float2 v[2];
                int nb[2][4];
                float wj[2][4], ai[2], be[2], mFF[2], mBB[2], nFB[2], Ic[2];
                bool mine[2], red[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = lane + 32 * u;
                    mine[u] = i < n;
                    const int ii = mine[u] ? i : 0;
                    const int x = ii % w, y = ii / w;
                    red[u] = ((x + y) & 1) == 0;
                    // starting F, B: nearest resize of the previous level
                    v[u] = src[nearest_src(y, ph, h) * pw + nearest_src(x, pw, w)];
                    nb[u][0] = y * w + max(x - 1, 0);
                    nb[u][1] = y * w + min(x + 1, w - 1);
                    nb[u][2] = max(y - 1, 0) * w + x;
                    nb[u][3] = min(y + 1, h - 1) * w + x;
                    ai[u] = Alv[o + ii];
                    be[u] = 1.f - ai[u];
                    float S = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        wj[u][j] = fmaf(p.omega, fabsf(ai[u] - Alv[o + nb[u][j]]), p.eps);
                        S += wj[u][j];
                    }
                    const float A00 = fmaf(ai[u], ai[u], S), A11 = fmaf(be[u], be[u], S);
                    const float A01 = ai[u] * be[u];
                    const float m = __fdividef(1.f, fmaf(A00, A11, -A01 * A01));
                    mFF[u] = A11 * m;
                    mBB[u] = A00 * m;
                    nFB[u] = -A01 * m;
                    Ic[u] = Ilv[3 * (o + ii) + c];
                }
                // the (F, B) of pixel j, held by lane j % 32 in slot j / 32
                auto fetch = [&](int j) {
                    float2 a;
                    a.x = __shfl_sync(kFull32, v[0].x, j & 31);
                    a.y = __shfl_sync(kFull32, v[0].y, j & 31);
                    if (two) {
                        float2 b;
                        b.x = __shfl_sync(kFull32, v[1].x, j & 31);
                        b.y = __shfl_sync(kFull32, v[1].y, j & 31);
                        if (j >= 32) a = b;
                    }
                    return a;
                };
                auto solve = [&](int u) {
                    float2 sv = __fmul2_rn(f2(wj[u][0], wj[u][0]), fetch(nb[u][0]));
#pragma unroll
                    for (int j = 1; j < 4; ++j) sv = __ffma2_rn(f2(wj[u][j], wj[u][j]), fetch(nb[u][j]), sv);
                    const float bF = fmaf(ai[u], Ic[u], sv.x), bB = fmaf(be[u], Ic[u], sv.y);
                    float gF = fmaf(mFF[u], bF, nFB[u] * bB);
                    float gB = fmaf(mBB[u], bB, nFB[u] * bF);
                    if (CLAMP) {
                        gF = __saturatef(gF);
                        gB = __saturatef(gB);
                    }
                    return f2(gF, gB);
                };
                const int rounds = p.order == 1 ? 2 * k : k;
                for (int it = 0; it < rounds; ++it) {
                    // Jacobi: every pixel from the previous values; red-black: one colour
                    // per round, the other keeps its value
                    // every lane of the warp computes (the shuffles need them all), then
                    // keeps the solution only where its pixel is updated in this half-sweep
                    float2 nv[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const bool upd = p.order != 1 || red[u] == ((it & 1) == 0);
                        nv[u] = v[u];
                        if (u == 0 || two) {
                            const float2 sol = solve(u);
                            if (upd) nv[u] = sol;
                        }
                    }
                    v[0] = nv[0];
                    v[1] = nv[1];
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (mine[u]) dst[lane + 32 * u] = v[u];
            }
            cur ^= 1;
            pw = w;
            ph = h;
            continue;
        }
        const int nt = (n + 31) & ~31;             // threads taking part in the barriers
        if (tid < nt) {
            // thread = pixel i, all three channels
            const bool mine = tid < n;
            const int i = mine ? tid : 0;
            const int x = i % w, y = i / w;
            float2 *src = buf + cur * 3 * kCoarseCap;
            float2 *dst = buf + (cur ^ 1) * 3 * kCoarseCap;
            // starting F, B: nearest resize of the previous level
            if (mine) {
                const int q = nearest_src(y, ph, h) * pw + nearest_src(x, pw, w);
#pragma unroll
                for (int c = 0; c < 3; ++c) dst[c * kCoarseCap + i] = src[c * kCoarseCap + q];
            }
            // neighbours clamped onto the level (Algorithm 1), their weights and A^{-1}
            int nb[4];
            nb[0] = y * w + max(x - 1, 0);
            nb[1] = y * w + min(x + 1, w - 1);
            nb[2] = max(y - 1, 0) * w + x;
            nb[3] = min(y + 1, h - 1) * w + x;
            const float ai = Alv[o + i], be = 1.f - ai;
            float wj[4], S = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                wj[j] = fmaf(p.omega, fabsf(ai - Alv[o + nb[j]]), p.eps);
                S += wj[j];
            }
            const float A00 = fmaf(ai, ai, S), A11 = fmaf(be, be, S), A01 = ai * be;
            const float m = __fdividef(1.f, fmaf(A00, A11, -A01 * A01));
            const float mFF = A11 * m, mBB = A00 * m, nFB = -A01 * m;
            float Ic[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) Ic[c] = Ilv[3 * (o + i) + c];
            cur ^= 1;
            level_sync(nt);

            auto solve = [&](float2 sv, float Icc) {
                const float bF = fmaf(ai, Icc, sv.x), bB = fmaf(be, Icc, sv.y);
                float gF = fmaf(mFF, bF, nFB * bB);
                float gB = fmaf(mBB, bB, nFB * bF);
                if (CLAMP) {
                    gF = __saturatef(gF);
                    gB = __saturatef(gB);
                }
                return f2(gF, gB);
            };
            if (p.order == 1) {
                // red-black: per iteration the x + y even pixels, then the odd ones, each
                // colour in place (it reads only the other colour, or itself at a border)
                const bool on0 = mine && ((x + y) & 1) == 0, on1 = mine && ((x + y) & 1) == 1;
                float2 *st = buf + cur * 3 * kCoarseCap;
                for (int it = 0; it < 2 * k; ++it) {
                    if ((it & 1) ? on1 : on0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float2 sv = __fmul2_rn(f2(wj[0], wj[0]), st[c * kCoarseCap + nb[0]]);
#pragma unroll
                            for (int j = 1; j < 4; ++j)
                                sv = __ffma2_rn(f2(wj[j], wj[j]), st[c * kCoarseCap + nb[j]], sv);
                            st[c * kCoarseCap + i] = solve(sv, Ic[c]);
                        }
                    }
                    level_sync(nt);
                }
            } else {
                for (int it = 0; it < k; ++it) {
                    const float2 *s2 = buf + cur * 3 * kCoarseCap;
                    float2 *d2 = buf + (cur ^ 1) * 3 * kCoarseCap;
                    if (mine) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            // (sum s_j F_j, sum s_j B_j) as one packed pair
                            float2 sv = __fmul2_rn(f2(wj[0], wj[0]), s2[c * kCoarseCap + nb[0]]);
#pragma unroll
                            for (int j = 1; j < 4; ++j)
                                sv = __ffma2_rn(f2(wj[j], wj[j]), s2[c * kCoarseCap + nb[j]], sv);
                            d2[c * kCoarseCap + i] = solve(sv, Ic[c]);
                        }
                    }
                    cur ^= 1;
                    level_sync(nt);
                }
            }
        } else {
            // the working threads swapped once for the resize and (Jacobi) once per sweep
            cur ^= p.order == 1 ? 1 : (k + 1) & 1;
        }
        pw = w;
        ph = h;
    }
    if (sizeof(T) == 4 && !rest_waited) cp_async_wait<0>();
    __syncthreads();

    const float2 *fin = buf + cur * 3 * kCoarseCap;
    T *F = static_cast<T *>(p.Fd);
    T *B = static_cast<T *>(p.Bd);
    if (tid < pw * ph) {
        const int x = tid % pw, y = tid / pw;
        float Fv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 v = fin[c * kCoarseCap + tid];
            Fv[c] = v.x;
            st_elem(F + (long long)y * p.d_pitch + 3 * x + c, v.x);
            st_elem(B + (long long)y * p.d_pitch + 3 * x + c, v.y);
        }
        if (p.In)
            composite_px<T>(p.Bn, p.bn_pitch, p.In, p.in_pitch, x, y,
                            Alv[p.off[p.nlev - 1] + tid], Fv);
    }
}

template <typename T, bool CLAMP>
cudaError_t launch_t(const CoarseArgs &a, cudaStream_t s) {
    const size_t smem = coarse_smem_bytes(a.total);
    cudaError_t e = allow_dynamic_smem(coarse_kernel<T, CLAMP>);
    if (e != cudaSuccess) return e;
    return launch_pdl(coarse_kernel<T, CLAMP>, dim3(1), dim3(kThreads), smem, s, a);
}

template <typename T, bool CLAMP>
cudaError_t launch_batch_t(const CoarseArgs *list, int n, int max_total, cudaStream_t s) {
    const size_t smem = coarse_smem_bytes(max_total);
    cudaError_t e = allow_dynamic_smem(coarse_batch_kernel<T, CLAMP>);
    if (e != cudaSuccess) return e;
    coarse_batch_kernel<T, CLAMP><<<n, kThreads, smem, s>>>(list);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_coarse_batch(int dtype, int clamp, const CoarseArgs *list, int n,
                                int max_total, cudaStream_t s) {
    if (n < 1 || max_total > kCoarseTotal) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return clamp ? launch_batch_t<float, true>(list, n, max_total, s) : launch_batch_t<float, false>(list, n, max_total, s);
        case kBF16:
            return clamp ? launch_batch_t<__nv_bfloat16, true>(list, n, max_total, s)
                         : launch_batch_t<__nv_bfloat16, false>(list, n, max_total, s);
        case kF16: return clamp ? launch_batch_t<__half, true>(list, n, max_total, s) : launch_batch_t<__half, false>(list, n, max_total, s);
    }
    return cudaErrorInvalidValue;
}

size_t coarse_smem_bytes(int total_pixels) {
    return 2 * 3 * kCoarseCap * sizeof(float2) + (size_t)total_pixels * 4 * sizeof(float);
}

cudaError_t launch_coarse(int dtype, int clamp, const CoarseArgs &a, cudaStream_t s) {
    if (a.nlev < 1 || a.nlev > kCoarseMaxLevels || a.total > kCoarseTotal) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return clamp ? launch_t<float, true>(a, s) : launch_t<float, false>(a, s);
        case kBF16:
            return clamp ? launch_t<__nv_bfloat16, true>(a, s) : launch_t<__nv_bfloat16, false>(a, s);
        case kF16: return clamp ? launch_t<__half, true>(a, s) : launch_t<__half, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
