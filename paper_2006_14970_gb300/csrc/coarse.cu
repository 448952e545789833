// Coarse levels: every level of at most 1024 pixels (with the paper's schedule, all
// the 10-sweep levels up to 32 x 32, Section III-D) runs inside one persistent
// 1024-thread block, one pixel per thread, from the 1x1 start of Algorithm 1 up to level
// `nlev`.
//  - I_l and alpha_l of every coarse level are gathered from the full-resolution input
//    (nearest resize, Algorithm 1) in one burst at the start, so HBM latency is paid once.
//  - F and B live in shared memory as (F, B) pairs per channel, ping-ponged between two
//    buffers, with one block barrier per Jacobi sweep.
//  - Each thread forms its pixel's neighbour weights and the inverse of its 2x2 matrix
//    (Section III-C) once per level; a sweep is then 4 neighbour reads, packed
//    multiply-adds and the clamped solve (Algorithm 1).
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 1024;

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

template <typename T, bool CLAMP>
__device__ __forceinline__ void coarse_body(const CoarseArgs &p);

template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads, 1) coarse_kernel(const CoarseArgs p) {
    pdl_enter();
    coarse_body<T, CLAMP>(p);
    pdl_leave();
}

// One block per image of a batch; each reads its arguments from the device list.
template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads, 1) coarse_batch_kernel(const CoarseArgs *list) {
    coarse_body<T, CLAMP>(list[blockIdx.x]);
}

template <typename T, bool CLAMP>
__device__ __forceinline__ void coarse_body(const CoarseArgs &p) {
    extern __shared__ __align__(16) float sm[];
    // [0, 3 * kCoarseCap) float2: buffer X; then buffer Y; then per level I (3 floats per
    // pixel) and alpha, at the offsets p.off[l] (in pixels)
    float2 *bufX = reinterpret_cast<float2 *>(sm);
    float2 *bufY = bufX + 3 * kCoarseCap;
    float *Ilv = reinterpret_cast<float *>(bufY + 3 * kCoarseCap);
    float *Alv = Ilv + 3 * p.total;
    const T *I = static_cast<const T *>(p.I);
    const T *A = static_cast<const T *>(p.A);
    const int tid = threadIdx.x;

    // gather I_l and alpha_l of all coarse levels: every load issued before any store
    constexpr int kPer = kCoarseTotal / kThreads;
    float gI[kPer][3], gA[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int idx = tid + k * kThreads;
        if (idx < p.total) {
            int l = 0;
            while (l + 1 < p.nlev && p.off[l + 1] <= idx) ++l;
            const int w = p.lw[l], h = p.lh[l], i = idx - p.off[l];
            const int x = i % w, y = i / w;
            const int gx = nearest_src(x, p.Iw, w), gy = nearest_src(y, p.Ih, h);
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
    float2 *cur = bufX, *nxt = bufY;
    if (tid == 0)
        for (int c = 0; c < 3; ++c) cur[c * kCoarseCap] = f2(p.init, p.init);   // 1 x 1 start
    __syncthreads();

    int pw = 1, ph = 1;
    for (int l = 0; l < p.nlev; ++l) {
        const int w = p.lw[l], h = p.lh[l], k = p.lk[l], n = w * h, o = p.off[l];
        const bool mine = tid < n;
        const int x = mine ? tid % w : 0, y = mine ? tid / w : 0;
        // starting F, B: nearest resize of the previous level
        if (mine) {
            const int q = nearest_src(y, ph, h) * pw + nearest_src(x, pw, w);
#pragma unroll
            for (int c = 0; c < 3; ++c) nxt[c * kCoarseCap + tid] = cur[c * kCoarseCap + q];
        }
        // neighbours clamped onto the level (Algorithm 1), their weights and A^{-1}
        int nb[4] = {0, 0, 0, 0};
        float wj[4] = {0.f, 0.f, 0.f, 0.f};
        float ai = 0.f, be = 0.f, mFF = 0.f, mBB = 0.f, nFB = 0.f, Ic[3] = {0.f, 0.f, 0.f};
        if (mine) {
            nb[0] = y * w + max(x - 1, 0);
            nb[1] = y * w + min(x + 1, w - 1);
            nb[2] = max(y - 1, 0) * w + x;
            nb[3] = min(y + 1, h - 1) * w + x;
            ai = Alv[o + tid];
            be = 1.f - ai;
            float S = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                wj[j] = fmaf(p.omega, fabsf(ai - Alv[o + nb[j]]), p.eps);
                S += wj[j];
            }
            const float A00 = fmaf(ai, ai, S), A11 = fmaf(be, be, S), A01 = ai * be;
            const float m = __fdividef(1.f, fmaf(A00, A11, -A01 * A01));
            mFF = A11 * m;
            mBB = A00 * m;
            nFB = -A01 * m;
#pragma unroll
            for (int c = 0; c < 3; ++c) Ic[c] = Ilv[3 * (o + tid) + c];
        }
        __syncthreads();
        { float2 *t = cur; cur = nxt; nxt = t; }

        for (int it = 0; it < k; ++it) {
            if (mine) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // (sum s_j F_j, sum s_j B_j) as one packed pair
                    float2 s = __fmul2_rn(f2(wj[0], wj[0]), cur[c * kCoarseCap + nb[0]]);
#pragma unroll
                    for (int j = 1; j < 4; ++j)
                        s = __ffma2_rn(f2(wj[j], wj[j]), cur[c * kCoarseCap + nb[j]], s);
                    const float bF = fmaf(ai, Ic[c], s.x), bB = fmaf(be, Ic[c], s.y);
                    float gF = fmaf(mFF, bF, nFB * bB);
                    float gB = fmaf(mBB, bB, nFB * bF);
                    if (CLAMP) {
                        gF = __saturatef(gF);
                        gB = __saturatef(gB);
                    }
                    nxt[c * kCoarseCap + tid] = f2(gF, gB);
                }
            }
            __syncthreads();
            { float2 *t = cur; cur = nxt; nxt = t; }
        }
        pw = w;
        ph = h;
    }

    T *F = static_cast<T *>(p.Fd);
    T *B = static_cast<T *>(p.Bd);
    if (tid < pw * ph) {
        const int x = tid % pw, y = tid / pw;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 v = cur[c * kCoarseCap + tid];
            st_elem(F + (long long)y * p.d_pitch + 3 * x + c, v.x);
            st_elem(B + (long long)y * p.d_pitch + 3 * x + c, v.y);
        }
    }
}

template <typename T, bool CLAMP>
cudaError_t launch_t(const CoarseArgs &a, cudaStream_t s) {
    const size_t smem = coarse_smem_bytes(a.total);
    cudaError_t e = cudaFuncSetAttribute(coarse_kernel<T, CLAMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(coarse_kernel<T, CLAMP>, dim3(1), dim3(kThreads), smem, s, a);
}

template <typename T, bool CLAMP>
cudaError_t launch_batch_t(const CoarseArgs *list, int n, int max_total, cudaStream_t s) {
    const size_t smem = coarse_smem_bytes(max_total);
    cudaError_t e = cudaFuncSetAttribute(coarse_batch_kernel<T, CLAMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
