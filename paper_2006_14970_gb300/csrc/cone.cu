// Small levels in one launch. Above the coarse kernel's levels, each level of a solve up to
// about 0.3 Mpx used to be one latency-bound launch (a few microseconds of work behind a
// launch, a gather and a write). Here the whole run of such levels is one launch.
//
// Each 256-thread block owns a 32 x 16 tile of the run's last level and computes, in shared
// memory, every level of the run on just the region its tile depends on. A level's k
// Jacobi sweeps (Algorithm 1) change a cell from its 4 neighbours only, so the tile after
// k sweeps depends on the start state over the tile expanded by k cells (clipped at the
// level's borders, where the clamped neighbour is the cell itself); that start state is
// the nearest resize of the level below (Algorithm 1), so it depends on the source range
// of the expanded region there, and so on down to the level the coarse kernel wrote. The
// block first gathers I and alpha of every level's region (nearest resize of the
// full-resolution input) — before it waits for the coarse kernel, which releases this
// launch as it starts, so the gathers overlap the coarse levels — then loads the bottom
// region of the state, and for each level resizes the level below into the expanded
// region and runs the sweeps on a region that shrinks by one cell per sweep on every side
// not at the level's border (the cells whose neighbours are all still exact), ending on a
// region that covers what the next level reads. Between levels the state is rounded to the
// storage type, as the per-level kernels store it. The per-pixel solve is the closed form
// of Section III-C with the same operation order as the small-level kernel, clamped to
// [0, 1]. Neighbouring blocks recompute the overlap of their regions; at the lower levels
// of a run that is most of the work, but those levels are tiny.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 256;

template <typename T> __device__ __forceinline__ float round_to(float v);
template <> __device__ __forceinline__ float round_to<float>(float v) { return v; }
template <> __device__ __forceinline__ float round_to<__nv_bfloat16>(float v) {
    return __bfloat162float(__float2bfloat16(v));
}
template <> __device__ __forceinline__ float round_to<__half>(float v) {
    return __half2float(__float2half(v));
}

template <typename T, bool CLAMP>
__global__ void __launch_bounds__(kThreads) cone_kernel(const ConeArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ ConeRect E[kConeMaxLevels];
    __shared__ ConeRect Rc;
    const int cap = a.cap;
    __shared__ int off[kConeMaxLevels];   // first cell of each level in the alpha/I area
    // two state buffers (6 channels each: F then B), then per level alpha and I (3
    // channels) of its region; a level's cells are indexed in the frame of its region E[l],
    // row-major
    float *P = sm, *Q = sm + 6 * cap;
    float *const io = sm + 12 * cap;
    const int tid = threadIdx.x;
    if (tid == 0) {
        cone_regions(a, blockIdx.x, blockIdx.y, E, &Rc);
        int o = 0;
        for (int l = 0; l < a.nlev; ++l) {
            off[l] = o;
            o += 4 * (E[l].x1 - E[l].x0 + 1) * (E[l].y1 - E[l].y0 + 1);
        }
    }
    __syncthreads();
    const T *I = static_cast<const T *>(a.I);
    const T *A = static_cast<const T *>(a.A);

    // alpha and I of every level's region, requested before the wait for the coarse
    // kernel: they are the solve's inputs, complete before the coarse kernel (which
    // writes only the state read below) was let through its own wait and released this
    // launch
    for (int l = 0; l < a.nlev; ++l) {
        const ConeRect e = E[l];
        const int w = a.lw[l], h = a.lh[l];
        const int ew = e.x1 - e.x0 + 1, n = ew * (e.y1 - e.y0 + 1);
        float *al = io + off[l], *im = al + n;
        for (int i = tid; i < n; i += kThreads) {
            const int xx = i % ew, yy = i / ew;
            const int gx = nearest_src(e.x0 + xx, a.Iw, w), gy = nearest_src(e.y0 + yy, a.Ih, h);
            al[i] = ld_elem(A + (long long)gy * a.A_pitch + gx);
            const T *Ip = I + (long long)gy * a.I_pitch + 3 * gx;
#pragma unroll
            for (int c = 0; c < 3; ++c) im[c * n + i] = ld_elem(Ip + c);
        }
    }
    pdl_enter();

    // the region of the level below the run, as the coarse kernel left it
    ConeRect pf = Rc;
    {
        const T *Fs = static_cast<const T *>(a.Fs);
        const T *Bs = static_cast<const T *>(a.Bs);
        const int pw = pf.x1 - pf.x0 + 1, n = pw * (pf.y1 - pf.y0 + 1);
        for (int i = tid; i < n; i += kThreads) {
            const int x = pf.x0 + i % pw, y = pf.y0 + i / pw;
            const T *Fp = Fs + (long long)y * a.s_pitch + 3 * x;
            const T *Bp = Bs + (long long)y * a.s_pitch + 3 * x;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                P[c * cap + i] = ld_elem(Fp + c);
                P[(3 + c) * cap + i] = ld_elem(Bp + c);
            }
        }
    }

    for (int l = 0; l < a.nlev; ++l) {
        const int w = a.lw[l], h = a.lh[l], k = a.lk[l];
        const int pwl = l > 0 ? a.lw[l - 1] : a.sw, phl = l > 0 ? a.lh[l - 1] : a.sh;
        const ConeRect e = E[l];
        const int ew = e.x1 - e.x0 + 1, n = ew * (e.y1 - e.y0 + 1);
        const int pfw = pf.x1 - pf.x0 + 1;
        const float *sAl = io + off[l], *sIm = sAl + n;
        __syncthreads();   // P complete; nothing reads Q any more
        for (int i = tid; i < n; i += kThreads) {
            const int x = e.x0 + i % ew, y = e.y0 + i / ew;
            const int j = (nearest_src(y, phl, h) - pf.y0) * pfw + (nearest_src(x, pwl, w) - pf.x0);
#pragma unroll
            for (int c = 0; c < 6; ++c) Q[c * cap + i] = round_to<T>(P[c * cap + j]);
        }
        {
            float *t = P;
            P = Q;
            Q = t;
        }
        ConeRect v = e;   // cells of P that hold this level's current iterate
        for (int t = 0; t < k; ++t) {
            __syncthreads();
            const ConeRect nv{v.x0 > 0 ? v.x0 + 1 : 0, v.y0 > 0 ? v.y0 + 1 : 0,
                              v.x1 < w - 1 ? v.x1 - 1 : v.x1, v.y1 < h - 1 ? v.y1 - 1 : v.y1};
            const int nw = nv.x1 - nv.x0 + 1, nn = nw * (nv.y1 - nv.y0 + 1);
            for (int i = tid; i < nn; i += kThreads) {
                const int x = nv.x0 + i % nw, y = nv.y0 + i / nw;
                const int c0 = (y - e.y0) * ew + (x - e.x0);
                const float ai = sAl[c0];
                const int nx[4] = {max(x - 1, 0), min(x + 1, w - 1), x, x};
                const int ny[4] = {y, y, max(y - 1, 0), min(y + 1, h - 1)};
                float S = 0.f, sF[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int o = (ny[q] - e.y0) * ew + (nx[q] - e.x0);
                    const float d = fmaf(a.omega, fabsf(ai - sAl[o]), a.eps);
                    S += d;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sF[c] = fmaf(d, P[c * cap + o], sF[c]);
                        sB[c] = fmaf(d, P[(3 + c) * cap + o], sB[c]);
                    }
                }
                const float be = 1.f - ai;
                const float A00 = fmaf(ai, ai, S), A11 = fmaf(be, be, S), A01 = ai * be;
                const float m = __fdividef(1.f, fmaf(A00, A11, -A01 * A01));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float Ic = sIm[c * n + c0];
                    const float bF = fmaf(ai, Ic, sF[c]), bB = fmaf(be, Ic, sB[c]);
                    float gF = (A11 * bF - A01 * bB) * m;
                    float gB = (A00 * bB - A01 * bF) * m;
                    if (CLAMP) {
                        gF = __saturatef(gF);
                        gB = __saturatef(gB);
                    }
                    Q[c * cap + c0] = gF;
                    Q[(3 + c) * cap + c0] = gB;
                }
            }
            float *tmp = P;
            P = Q;
            Q = tmp;
            v = nv;
        }
        pf = e;
    }
    __syncthreads();

    // the block's tile of the run's last level
    const int L = a.nlev - 1;
    const ConeRect e = E[L];
    const int ew = e.x1 - e.x0 + 1;
    const int X0 = blockIdx.x * kConeTW, Y0 = blockIdx.y * kConeTH;
    T *Fd = static_cast<T *>(a.Fd);
    T *Bd = static_cast<T *>(a.Bd);
    for (int i = tid; i < kConeTW * kConeTH; i += kThreads) {
        const int x = X0 + i % kConeTW, y = Y0 + i / kConeTW;
        if (x >= a.lw[L] || y >= a.lh[L]) continue;
        const int c0 = (y - e.y0) * ew + (x - e.x0);
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = P[c * cap + c0];
        T *Fp = Fd + (long long)y * a.d_pitch + 3 * x;
        T *Bp = Bd + (long long)y * a.d_pitch + 3 * x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st_elem(Fp + c, v[c]);
            st_elem(Bp + c, v[3 + c]);
        }
        if (a.In) composite_px<T>(a.Bn, a.bn_pitch, a.In, a.in_pitch, x, y, io[off[L] + c0], v);
    }
    pdl_leave();
}

template <typename T, bool CLAMP>
cudaError_t launch_t(const ConeArgs &a, cudaStream_t s) {
    const int L = a.nlev - 1;
    const dim3 grid((a.lw[L] + kConeTW - 1) / kConeTW, (a.lh[L] + kConeTH - 1) / kConeTH);
    const size_t smem = cone_smem_bytes(a.cap, a.io);
    cudaError_t e = allow_dynamic_smem(cone_kernel<T, CLAMP>);
    if (e != cudaSuccess) return e;
    return launch_pdl(cone_kernel<T, CLAMP>, grid, dim3(kThreads), smem, s, a);
}

}  // namespace

size_t cone_smem_bytes(int cap, int io) { return ((size_t)cap * 12 + (size_t)io * 4) * sizeof(float); }

cudaError_t launch_cone(int dtype, int clamp, const ConeArgs &a, cudaStream_t s) {
    if (a.nlev < 1 || a.nlev > kConeMaxLevels || a.cap < 1 || a.io < 1) return cudaErrorInvalidValue;
    if ((a.lh[a.nlev - 1] + kConeTH - 1) / kConeTH > 65535) return cudaErrorInvalidValue;
    switch (dtype) {
        case kF32: return clamp ? launch_t<float, true>(a, s) : launch_t<float, false>(a, s);
        case kBF16:
            return clamp ? launch_t<__nv_bfloat16, true>(a, s) : launch_t<__nv_bfloat16, false>(a, s);
        case kF16: return clamp ? launch_t<__half, true>(a, s) : launch_t<__half, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
