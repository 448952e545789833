// Coarse levels: every level whose F and B fit in one SM's shared memory runs inside
// one persistent 1024-thread block, from the 1x1 start of Algorithm 1 up to level
// `nlev`. Only the level's I values and alpha come from HBM (nearest resize of the
// full-resolution input, Algorithm 1); the starting F and B of a level are the nearest
// resize of the previous level, done shared memory to shared memory, and the sweeps
// (10 per small level, Section III-D) ping-pong between two shared buffers with a block
// barrier per Jacobi sweep. The per-pixel solve is the closed form of Section III-C,
// as in the level-pass kernel, in scalar float32.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 1024;

// Shared memory: two F/B buffers (6 planes each), alpha, and a packed (row, column)
// source index of I per pixel.
constexpr size_t kSmemBytes = (size_t)kCoarseCap * (13 * sizeof(float) + sizeof(int));

template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads, 1) coarse_kernel(const CoarseArgs p) {
    extern __shared__ float sm[];
    float *bufA = sm;
    float *bufB = sm + 6 * kCoarseCap;
    float *al = sm + 12 * kCoarseCap;
    int *isrc = reinterpret_cast<int *>(sm + 13 * kCoarseCap);
    const T *I = static_cast<const T *>(p.I);
    const T *A = static_cast<const T *>(p.A);
    const int tid = threadIdx.x;

    float *cur = bufA, *nxt = bufB;
    if (tid < 6) cur[tid * kCoarseCap] = p.init;     // F, B <- init at 1 x 1
    int pw = 1, ph = 1;
    __syncthreads();

    for (int l = 0; l < p.nlev; ++l) {
        const int w = p.lw[l], h = p.lh[l], k = p.lk[l], n = w * h;
        // resize: alpha and the I source index from the full-resolution input,
        // F and B from the previous level
        for (int i = tid; i < n; i += kThreads) {
            const int x = i % w, y = i / w;
            const int gx = nearest_src(x, p.Iw, w), gy = nearest_src(y, p.Ih, h);
            isrc[i] = (gy << 16) | gx;
            al[i] = ld_elem(A + (long long)gy * p.A_pitch + gx);
            const int q = nearest_src(y, ph, h) * pw + nearest_src(x, pw, w);
#pragma unroll
            for (int c = 0; c < 6; ++c) nxt[c * kCoarseCap + i] = cur[c * kCoarseCap + q];
        }
        __syncthreads();
        { float *t = cur; cur = nxt; nxt = t; }

        for (int it = 0; it < k; ++it) {
            for (int i = tid; i < n; i += kThreads) {
                const int x = i % w, y = i / w;
                const float ai = al[i];
                // the 4 neighbours, clamped onto the image (Algorithm 1)
                const int nb[4] = {y * w + max(x - 1, 0), y * w + min(x + 1, w - 1),
                                   max(y - 1, 0) * w + x, min(y + 1, h - 1) * w + x};
                float S = 0.f;
                float sF[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = nb[j];
                    const float d = fmaf(p.omega, fabsf(ai - al[q]), p.eps);
                    S += d;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sF[c] = fmaf(d, cur[c * kCoarseCap + q], sF[c]);
                        sB[c] = fmaf(d, cur[(3 + c) * kCoarseCap + q], sB[c]);
                    }
                }
                const int src = isrc[i];
                const T *Ip = I + (long long)(src >> 16) * p.I_pitch + 3 * (src & 0xffff);
                const float be = 1.f - ai;
                const float A00 = fmaf(ai, ai, S), A11 = fmaf(be, be, S), A01 = ai * be;
                const float m = __frcp_rn(fmaf(A00, A11, -A01 * A01));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float Ic = ld_elem(Ip + c);
                    const float bF = fmaf(ai, Ic, sF[c]), bB = fmaf(be, Ic, sB[c]);
                    float gF = (A11 * bF - A01 * bB) * m;
                    float gB = (A00 * bB - A01 * bF) * m;
                    if (CLAMP) {
                        gF = __saturatef(gF);
                        gB = __saturatef(gB);
                    }
                    nxt[c * kCoarseCap + i] = gF;
                    nxt[(3 + c) * kCoarseCap + i] = gB;
                }
            }
            __syncthreads();
            { float *t = cur; cur = nxt; nxt = t; }
        }
        pw = w;
        ph = h;
    }

    T *F = static_cast<T *>(p.Fd);
    T *B = static_cast<T *>(p.Bd);
    for (int i = tid; i < pw * ph; i += kThreads) {
        const int x = i % pw, y = i / pw;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st_elem(F + (long long)y * p.d_pitch + 3 * x + c, cur[c * kCoarseCap + i]);
            st_elem(B + (long long)y * p.d_pitch + 3 * x + c, cur[(3 + c) * kCoarseCap + i]);
        }
    }
}

template <typename T, bool CLAMP>
cudaError_t launch_t(const CoarseArgs &a, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(coarse_kernel<T, CLAMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    coarse_kernel<T, CLAMP><<<1, kThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t coarse_smem_bytes() { return kSmemBytes; }

cudaError_t launch_coarse(int dtype, int clamp, const CoarseArgs &a, cudaStream_t s) {
    switch (dtype) {
        case kF32: return clamp ? launch_t<float, true>(a, s) : launch_t<float, false>(a, s);
        case kBF16:
            return clamp ? launch_t<__nv_bfloat16, true>(a, s) : launch_t<__nv_bfloat16, false>(a, s);
        case kF16: return clamp ? launch_t<__half, true>(a, s) : launch_t<__half, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
