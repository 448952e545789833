// Small levels: K <= 2 Jacobi sweeps of a level with few pixels, where the row-streaming
// kernels are bound by the latency of their row-by-row walk. One 256-thread block owns a
// 32 x 16 tile of outputs: it gathers the tile plus a K-pixel halo in one burst (alpha and
// I by nearest resize of the full-resolution input, F and B by nearest resize of the
// starting state, Algorithm 1), runs the sweeps in shared memory with one barrier
// between them, and writes the tile. Neighbours are clamped onto the image as in
// Algorithm 1, so a halo cell outside the image is never read. The per-pixel solve is
// the closed form of Section III-C, clamped to [0, 1].
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kTW = 32, kTH = 16, kThreads = 256;

template <typename T, int K, bool CLAMP>
__global__ void __launch_bounds__(kThreads) level_small_kernel(const PassArgs p) {
    constexpr int RW = kTW + 2 * K, RH = kTH + 2 * K, RN = RW * RH;   // gathered region
    constexpr int W1 = kTW + 2 * (K - 1), H1 = kTH + 2 * (K - 1);     // sweep-1 region
    constexpr int CPT = (RN + kThreads - 1) / kThreads;
    __shared__ float sA[RN];
    __shared__ float sI[3][RN];
    __shared__ float s0[6][RN];                                       // starting F, B
    __shared__ float s1[6][K == 2 ? W1 * H1 : 1];                     // after sweep 1
    pdl_enter();

    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kTW, Y0 = blockIdx.y * kTH;
    const int RX = X0 - K, RY = Y0 - K;   // image coordinates of region cell (0, 0)
    const T *I = static_cast<const T *>(p.I);
    const T *A = static_cast<const T *>(p.A);
    const T *Fs = static_cast<const T *>(p.Fs);
    const T *Bs = static_cast<const T *>(p.Bs);

    // gather: every load of the region issued before any is stored
    float va[CPT], vi[CPT][3], vf[CPT][6];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int idx = tid + k * kThreads;
        if (idx < RN) {
            const int x = min(max(RX + idx % RW, 0), p.w - 1);
            const int y = min(max(RY + idx / RW, 0), p.h - 1);
            const int gx = nearest_src(x, p.Iw, p.w), gy = nearest_src(y, p.Ih, p.h);
            const int sx = nearest_src(x, p.sw, p.w), sy = nearest_src(y, p.sh, p.h);
            const T *Ip = I + (long long)gy * p.I_pitch + 3 * gx;
            const T *Fp = Fs + (long long)sy * p.s_pitch + 3 * sx;
            const T *Bp = Bs + (long long)sy * p.s_pitch + 3 * sx;
            va[k] = ld_elem(A + (long long)gy * p.A_pitch + gx);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                vi[k][c] = ld_elem(Ip + c);
                vf[k][c] = ld_elem(Fp + c);
                vf[k][3 + c] = ld_elem(Bp + c);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int idx = tid + k * kThreads;
        if (idx < RN) {
            sA[idx] = va[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) sI[c][idx] = vi[k][c];
#pragma unroll
            for (int c = 0; c < 6; ++c) s0[c][idx] = vf[k][c];
        }
    }
    __syncthreads();

    // one update of the cell at image (x, y); `src` holds the previous state over a
    // window whose cell (0, 0) is image (ox, oy) and whose width is sw_
    auto solve = [&](int x, int y, const auto &src, int ox, int oy, int swid, float *outv) {
        const int i = (y - RY) * RW + (x - RX);
        const float ai = sA[i];
        const int nx[4] = {max(x - 1, 0), min(x + 1, p.w - 1), x, x};
        const int ny[4] = {y, y, max(y - 1, 0), min(y + 1, p.h - 1)};
        float S = 0.f, sF[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float d = fmaf(p.omega, fabsf(ai - sA[(ny[j] - RY) * RW + (nx[j] - RX)]), p.eps);
            const int o = (ny[j] - oy) * swid + (nx[j] - ox);
            S += d;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sF[c] = fmaf(d, src[c][o], sF[c]);
                sB[c] = fmaf(d, src[3 + c][o], sB[c]);
            }
        }
        const float be = 1.f - ai;
        const float A00 = fmaf(ai, ai, S), A11 = fmaf(be, be, S), A01 = ai * be;
        const float m = __fdividef(1.f, fmaf(A00, A11, -A01 * A01));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float bF = fmaf(ai, sI[c][i], sF[c]), bB = fmaf(be, sI[c][i], sB[c]);
            float gF = (A11 * bF - A01 * bB) * m;
            float gB = (A00 * bB - A01 * bF) * m;
            if (CLAMP) {
                gF = __saturatef(gF);
                gB = __saturatef(gB);
            }
            outv[c] = gF;
            outv[3 + c] = gB;
        }
    };

    T *Fd = static_cast<T *>(p.Fd);
    T *Bd = static_cast<T *>(p.Bd);
    if (K == 2) {
        // sweep 1 over the tile plus one cell, inside the image
        for (int idx = tid; idx < W1 * H1; idx += kThreads) {
            const int x = X0 - 1 + idx % W1, y = Y0 - 1 + idx / W1;
            if (x < 0 || y < 0 || x >= p.w || y >= p.h) continue;
            float v[6];
            solve(x, y, s0, RX, RY, RW, v);
#pragma unroll
            for (int c = 0; c < 6; ++c) s1[c][idx] = v[c];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < kTW * kTH; idx += kThreads) {
        const int x = X0 + idx % kTW, y = Y0 + idx / kTW;
        if (x >= p.w || y >= p.h) continue;
        float v[6];
        if (K == 2)
            solve(x, y, s1, X0 - 1, Y0 - 1, W1, v);
        else
            solve(x, y, s0, RX, RY, RW, v);
        T *Fp = Fd + (long long)y * p.d_pitch + 3 * x;
        T *Bp = Bd + (long long)y * p.d_pitch + 3 * x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st_elem(Fp + c, v[c]);
            st_elem(Bp + c, v[3 + c]);
        }
        if (p.In)
            composite_px<T>(p.Bn, p.bn_pitch, p.In, p.in_pitch, x, y,
                            sA[(y - RY) * RW + (x - RX)], v);
    }
    pdl_leave();
}

template <typename T, int K, bool CLAMP>
cudaError_t launch_t(const PassArgs &a, cudaStream_t s) {
    const dim3 grid((a.w + kTW - 1) / kTW, (a.h + kTH - 1) / kTH);
    return launch_pdl(level_small_kernel<T, K, CLAMP>, grid, dim3(kThreads), 0, s, a);
}

template <typename T>
cudaError_t launch_dtype(int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if (iters == 1) return clamp ? launch_t<T, 1, true>(a, s) : launch_t<T, 1, false>(a, s);
    if (iters == 2) return clamp ? launch_t<T, 2, true>(a, s) : launch_t<T, 2, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_level_small(int dtype, int iters, int clamp, const PassArgs &a,
                               cudaStream_t s) {
    if ((long long)((a.h + kTH - 1) / kTH) > 65535) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return launch_dtype<float>(iters, clamp, a, s);
        case kBF16: return launch_dtype<__nv_bfloat16>(iters, clamp, a, s);
        case kF16: return launch_dtype<__half>(iters, clamp, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
