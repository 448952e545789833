// Red-black order: K <= 2 red-black iterations of a level, each a half-sweep over the
// pixels with x + y even followed by one over the pixels with x + y odd. A pixel of one
// colour reads only pixels of the other colour (or itself, at a clamped border), so each
// half-sweep may update its colour in place and the result is independent of the order
// inside it (the iteration of Algorithm 1 with the red-black visiting order).
//
// One 256-thread block owns a 32 x 16 tile of outputs. It gathers the tile plus a halo of
// 2K cells (alpha and I by nearest resize of the full-resolution input, F and B by
// nearest resize of the starting state, Algorithm 1), then runs the 2K half-sweeps in
// shared memory: half-sweep h updates its colour within distance 2K - h - 1 of the tile,
// the cells whose neighbours are all still exact, so the last one covers the tile
// itself. Neighbours are clamped onto the image (Algorithm 1); cells of the halo outside
// the image are never read. The per-pixel solve is the closed form of Section III-C,
// clamped to [0, 1].
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kTW = 32, kTH = 16, kThreads = 256;

template <typename T, int K, bool CLAMP>
__global__ void __launch_bounds__(kThreads) level_rb_kernel(const PassArgs p) {
    constexpr int H = 2 * K;                                   // one halo cell per half-sweep
    constexpr int RW = kTW + 2 * H, RH = kTH + 2 * H, RN = RW * RH;
    constexpr int CPT = (RN + kThreads - 1) / kThreads;
    __shared__ float sA[RN];
    __shared__ float sI[3][RN];
    __shared__ float sS[6][RN];                                // F (3), B (3), in place
    pdl_enter();

    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kTW, Y0 = blockIdx.y * kTH;
    const int RX = X0 - H, RY = Y0 - H;   // image coordinates of region cell (0, 0)
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
            for (int c = 0; c < 6; ++c) sS[c][idx] = vf[k][c];
        }
    }
    __syncthreads();

#pragma unroll 1
    for (int hs = 0; hs < 2 * K; ++hs) {
        const int colour = hs & 1;
        const int d = H - hs - 1;
        const int ux0 = max(X0 - d, 0), ux1 = min(X0 + kTW + d, p.w);
        const int uy0 = max(Y0 - d, 0), uy1 = min(Y0 + kTH + d, p.h);
        const int half = (ux1 - ux0 + 1) / 2;   // cells of one colour per row, at most
        for (int idx = tid; idx < half * (uy1 - uy0); idx += kThreads) {
            const int y = uy0 + idx / half;
            const int x = ux0 + ((ux0 + y + colour) & 1) + 2 * (idx % half);
            if (x >= ux1) continue;
            const int i = (y - RY) * RW + (x - RX);
            const float ai = sA[i];
            const int nx[4] = {max(x - 1, 0), min(x + 1, p.w - 1), x, x};
            const int ny[4] = {y, y, max(y - 1, 0), min(y + 1, p.h - 1)};
            float S = 0.f, sF[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = (ny[j] - RY) * RW + (nx[j] - RX);
                const float dj = fmaf(p.omega, fabsf(ai - sA[o]), p.eps);
                S += dj;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sF[c] = fmaf(dj, sS[c][o], sF[c]);
                    sB[c] = fmaf(dj, sS[3 + c][o], sB[c]);
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
                sS[c][i] = gF;
                sS[3 + c][i] = gB;
            }
        }
        __syncthreads();
    }

    T *Fd = static_cast<T *>(p.Fd);
    T *Bd = static_cast<T *>(p.Bd);
    for (int idx = tid; idx < kTW * kTH; idx += kThreads) {
        const int x = X0 + idx % kTW, y = Y0 + idx / kTW;
        if (x >= p.w || y >= p.h) continue;
        const int i = (y - RY) * RW + (x - RX);
        T *Fp = Fd + (long long)y * p.d_pitch + 3 * x;
        T *Bp = Bd + (long long)y * p.d_pitch + 3 * x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st_elem(Fp + c, sS[c][i]);
            st_elem(Bp + c, sS[3 + c][i]);
        }
        if (p.In) {
            const float F[3] = {sS[0][i], sS[1][i], sS[2][i]};
            composite_px<T>(p.Bn, p.bn_pitch, p.In, p.in_pitch, x, y, sA[i], F);
        }
    }
    pdl_leave();
}

template <typename T, int K, bool CLAMP>
cudaError_t launch_t(const PassArgs &a, cudaStream_t s) {
    const dim3 grid((a.w + kTW - 1) / kTW, (a.h + kTH - 1) / kTH);
    return launch_pdl(level_rb_kernel<T, K, CLAMP>, grid, dim3(kThreads), 0, s, a);
}

template <typename T>
cudaError_t launch_dtype(int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if (iters == 1) return clamp ? launch_t<T, 1, true>(a, s) : launch_t<T, 1, false>(a, s);
    if (iters == 2) return clamp ? launch_t<T, 2, true>(a, s) : launch_t<T, 2, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_level_rb(int dtype, int iters, int clamp, const PassArgs &a, cudaStream_t s) {
    if ((long long)((a.h + kTH - 1) / kTH) > 65535) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return launch_dtype<float>(iters, clamp, a, s);
        case kBF16: return launch_dtype<__nv_bfloat16>(iters, clamp, a, s);
        case kF16: return launch_dtype<__half>(iters, clamp, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
