// Error measures of the foreground estimate (Section IV-C): over the pixels with
// 0 < alpha_gt < 1, weighted by alpha_gt,
//   SAD = sum a |F_est - F_gt|_1, MSE = sum a |F_est - F_gt|_2^2,
//   GRAD = sum a |grad F_est - grad F_gt|_2^2,
// with the gradient taken by first-order Gaussian derivative filters (sigma = 1.4,
// taps k = -6..6, borders repeated). The filters are linear, so GRAD uses the gradient
// of the difference D = F_est - F_gt.
//
// One 256-thread block owns a 32 x 16 tile: it loads D over the tile plus a 6-pixel halo
// into shared memory (coordinates clamped onto the image, which repeats the border),
// filters the rows (derivative and smoothing taps) and then the columns, and reduces its
// pixels' three sums into one double-precision partial per block. A second one-block
// kernel adds the partials in a fixed order, so the result is deterministic.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kTW = 32, kTH = 16, kThreads = 256;
constexpr int R = kQualityRadius;
constexpr int RW = kTW + 2 * R, RH = kTH + 2 * R;

__device__ __forceinline__ double block_sum(double v, double *red) { return block_sum_d(v, red); }

template <typename T>
__global__ void __launch_bounds__(kThreads) quality_kernel(const QualityArgs q) {
    __shared__ float sD[3][RH][RW];
    __shared__ float sX[3][RH][kTW];   // rows filtered with the derivative taps
    __shared__ float sS[3][RH][kTW];   // rows filtered with the smoothing taps
    __shared__ double red[kThreads / 32];
    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kTW, Y0 = blockIdx.y * kTH;
    const T *Fe = static_cast<const T *>(q.Fe);
    const T *Fg = static_cast<const T *>(q.Fg);
    const T *A = static_cast<const T *>(q.A);

    for (int idx = tid; idx < RW * RH; idx += kThreads) {
        const int rx = idx % RW, ry = idx / RW;
        const int x = min(max(X0 - R + rx, 0), q.w - 1);
        const int y = min(max(Y0 - R + ry, 0), q.h - 1);
        const T *pe = Fe + (long long)y * q.fe_pitch + 3 * x;
        const T *pg = Fg + (long long)y * q.fg_pitch + 3 * x;
#pragma unroll
        for (int c = 0; c < 3; ++c) sD[c][ry][rx] = ld_elem(pe + c) - ld_elem(pg + c);
    }
    __syncthreads();
    // row pass: out[x] = sum_j tap(j) D[x - j], j = -R..R
    for (int idx = tid; idx < 3 * RH * kTW; idx += kThreads) {
        const int tx = idx % kTW, ry = (idx / kTW) % RH, c = idx / (kTW * RH);
        float vx = 0.f, vs = 0.f;
#pragma unroll
        for (int j = -R; j <= R; ++j) {
            const float d = sD[c][ry][tx + R - j];
            vx = fmaf(q.dg[j + R], d, vx);
            vs = fmaf(q.g[j + R], d, vs);
        }
        sX[c][ry][tx] = vx;
        sS[c][ry][tx] = vs;
    }
    __syncthreads();
    double sad = 0.0, mse = 0.0, grad = 0.0;
    for (int idx = tid; idx < kTW * kTH; idx += kThreads) {
        const int tx = idx % kTW, ty = idx / kTW;
        const int x = X0 + tx, y = Y0 + ty;
        if (x >= q.w || y >= q.h) continue;
        const float a = ld_elem(A + (long long)y * q.a_pitch + x);
        if (!(a > 0.f && a < 1.f)) continue;
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float gx = 0.f, gy = 0.f;
#pragma unroll
            for (int j = -R; j <= R; ++j) {
                gx = fmaf(q.g[j + R], sX[c][ty + R - j][tx], gx);
                gy = fmaf(q.dg[j + R], sS[c][ty + R - j][tx], gy);
            }
            const float d = sD[c][ty + R][tx + R];
            s1 += fabsf(d);
            s2 = fmaf(d, d, s2);
            s3 = fmaf(gx, gx, fmaf(gy, gy, s3));
        }
        sad += (double)a * s1;
        mse += (double)a * s2;
        grad += (double)a * s3;
    }
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    sad = block_sum(sad, red);
    if (tid == 0) q.partials[3 * b + 0] = sad;
    mse = block_sum(mse, red);
    if (tid == 0) q.partials[3 * b + 1] = mse;
    grad = block_sum(grad, red);
    if (tid == 0) q.partials[3 * b + 2] = grad;
}

__global__ void __launch_bounds__(kThreads) quality_sum_kernel(const double *partials, long long n,
                                                               double *out) {
    __shared__ double red[kThreads / 32];
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (long long i = threadIdx.x; i < n; i += kThreads) v += partials[3 * i + k];
        v = block_sum(v, red);
        if (threadIdx.x == 0) out[k] = v;
    }
}

}  // namespace

long long quality_blocks(int w, int h) {
    return (long long)((w + kTW - 1) / kTW) * ((h + kTH - 1) / kTH);
}

cudaError_t launch_quality(int dtype, const QualityArgs &q, double *out, cudaStream_t s) {
    const dim3 grid((q.w + kTW - 1) / kTW, (q.h + kTH - 1) / kTH);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: quality_kernel<float><<<grid, kThreads, 0, s>>>(q); break;
        case kBF16: quality_kernel<__nv_bfloat16><<<grid, kThreads, 0, s>>>(q); break;
        case kF16: quality_kernel<__half><<<grid, kThreads, 0, s>>>(q); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    quality_sum_kernel<<<1, kThreads, 0, s>>>(q.partials, quality_blocks(q.w, q.h), out);
    return cudaGetLastError();
}

}  // namespace fgml
