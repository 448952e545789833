// Internal declarations shared by the CUDA translation units of libfgml.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <algorithm>
#include <utility>

namespace fgml {

// ------------------------------------------------------------------ storage types
// Images are stored as float32, bfloat16 or float16; all arithmetic is float32.
template <typename T> __device__ __forceinline__ float ld_elem(const T *p);
template <> __device__ __forceinline__ float ld_elem<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_elem<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ld_elem<__half>(const __half *p) {
    return __half2float(__ldg(p));
}

template <typename T> __device__ __forceinline__ void st_elem(T *p, float v);
template <> __device__ __forceinline__ void st_elem<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void st_elem<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void st_elem<__half>(__half *p, float v) {
    *p = __float2half_rn(v);
}

// Centre-aligned nearest-neighbour source index of destination index d when a side of
// length S is resized to length D: floor((2d + 1) S / (2 D)). Sides are <= 32767, so the
// product fits in 32 bits.
__host__ __device__ __forceinline__ int nearest_src(int d, int S, int D) {
    return (int)(((2u * (unsigned)d + 1u) * (unsigned)S) / (2u * (unsigned)D));
}

// ------------------------------------------------------------------ kernel arguments
struct PassArgs {
    const void *I;          // full-resolution image, 3 channels per pixel
    long long I_pitch;      // elements per row
    const void *A;          // full-resolution alpha
    long long A_pitch;      // elements per row
    int Iw, Ih;             // full-resolution size
    const void *Fs, *Bs;    // starting F and B (previous level or previous pass)
    long long s_pitch;      // elements per row of Fs and Bs
    int sw, sh;             // size of Fs and Bs
    void *Fd, *Bd;          // output F and B of this level
    long long d_pitch;      // elements per row of Fd and Bd
    int w, h;               // level size
    float eps, omega;
    int strip_h;            // output rows per warp
    int n_xstrips;          // strips of 60 output columns
    int n_warps;            // n_xstrips * ceil(h / strip_h)
    // row-ring variant only: bytes of each segment of a ring slot (multiples of 16)
    int capI, capA, capS, slot_bytes;
    // row-ring variant only: one past the last byte of I, alpha, Fs and Bs
    const void *I_end, *A_end, *Fs_end, *Bs_end;
    // level_tile.cu: tensor-gather box widths (in elements of tile_u* bytes: 8, 4 or 2, the
    // largest unit that divides a row) of I, alpha and the starting F and B; chunk slots in
    // flight per warp, bytes of one chunk slot, bytes the gathers of one chunk deliver
    int tile_bwI, tile_bwA, tile_bwS, tile_slots;
    int tile_uI, tile_uA, tile_uS;
    int tile_chunk, tile_tx;
    // chunk pipeline of level_tile.cu, per image (0 I, 1 alpha, 2 F, 3 B): rows of the
    // image arrive by tensor gather (mode 0, box of tile_bw*/tile_u*) or by per-lane
    // asynchronous copies of the lane's own pixels (mode 1); lt_row = bytes of one row of
    // the image in a chunk slot, lt_off = offset of its rows in the slot
    int lt_mode[4], lt_row[4], lt_off[4];
    // optional compositing epilogue (In == nullptr: none): as the pass stores F it also
    // writes In = alpha F + (1 - alpha) Bn at the same pixel, alpha being the level's
    const void *Bn;         // new background, w x h x 3
    void *In;               // composite, w x h x 3
    long long bn_pitch, in_pitch;   // elements per row
};

// Compositing epilogue of one pixel (see PassArgs::In), channels c = 0..2 of F.
template <typename T>
__device__ __forceinline__ void composite_px(const void *Bn, long long bn_pitch, void *In,
                                             long long in_pitch, int x, int y, float a,
                                             const float *F) {
    const T *b = static_cast<const T *>(Bn) + (long long)y * bn_pitch + 3 * x;
    T *o = static_cast<T *>(In) + (long long)y * in_pitch + 3 * x;
#pragma unroll
    for (int c = 0; c < 3; ++c) st_elem(o + c, fmaf(a, F[c], (1.f - a) * ld_elem(b + c)));
}

// One level pass of a work-list batch.
struct TileMaps {
    CUtensorMap I, A, F, B;
};

struct BatchDesc {
    PassArgs a;
    int iters;       // sweeps of this pass (1 or 2)
    int dep;         // pass whose strips must all be done first (-1: none)
    int dep_count;   // strips of that pass
    TileMaps maps;   // the pass's tensor maps (64-byte aligned in the device array)
};

// One work item: strip `warp` of pass `desc`.
struct BatchItem {
    int desc, warp;
};

struct BatchLaunch {
    const BatchDesc *descs;
    const BatchItem *items;
    int n_items;
    int *counters;       // [0]: next item to pop, [1 + d]: finished strips of pass d
    long long wait_ns;   // bound of one dependency wait
    int slot_bytes;      // ring slot size (largest over the ring passes, >= 16)
    int region;          // shared-memory bytes per warp (ring slots or tile chunks)
    int blocks;          // persistent grid (at most the resident blocks)
};

// One row-aligned copy (stage.cu): `rows` rows of `row_bytes` from src (pitch src_pitch
// bytes) to dst (pitch dst_pitch, a multiple of 16; dst 16-byte aligned).
struct StageJob {
    const void *src;
    void *dst;
    long long src_pitch, dst_pitch, row_bytes, rows;
    long long row0;   // first row of this job among the rows of all jobs of the launch
};
// The jobs of one launch: a device array, or (dev == nullptr) up to two by value.
struct StageList {
    const StageJob *dev;
    StageJob local[2];
};
// Runs the jobs in one launch; total_rows = the rows of all jobs.
cudaError_t launch_stage_rows(int dtype, const StageList &list, int njobs, long long total_rows,
                              cudaStream_t s);


// Adds to *bad (device) the number of values of a w x h x ch image (pitch in elements)
// outside [0, 1] or NaN (the optional input check).
cudaError_t launch_range_check(int dtype, const void *p, long long pitch, int w, int h, int ch,
                               unsigned long long *bad, cudaStream_t s);


// Tensor maps of the tile variant: I, alpha, and the starting F and B, as 2D tensors of
// 8-byte elements (a row's bytes / 8), box one row high for gather-mode copies.
// Largest source-column span (in pixels) of one warp strip of a level pass, for a gather
// from a side of length S to a level side of length D (host planning of ring slots).
int strip_span(int S, int D);
// Per-warp ring slots of the row-ring level pass.
constexpr int kRingSlots = 6;

constexpr int kCoarseCap = 1024;     // pixels of the largest level the one-block kernel runs
constexpr int kCoarseMaxLevels = 16;
constexpr int kCoarseTotal = 8192;   // pixels of all its levels together

struct CoarseArgs {
    const void *I;
    long long I_pitch;
    const void *A;
    long long A_pitch;
    int Iw, Ih;
    int nlev;                              // levels 1..nlev run in the block
    int lw[kCoarseMaxLevels], lh[kCoarseMaxLevels], lk[kCoarseMaxLevels];
    int off[kCoarseMaxLevels];             // first pixel of each level in the gathered I/alpha
    int total;                             // pixels of all nlev levels
    void *Fd, *Bd;                         // F and B of level nlev
    long long d_pitch;
    float eps, omega, init;
    int order;                             // 0 Jacobi, 1 red-black
    const void *Bn;                        // compositing epilogue of level nlev, as PassArgs
    void *In;
    long long bn_pitch, in_pitch;
};

enum DType { kF32 = 0, kBF16 = 1, kF16 = 2 };

// Error measures (Section IV-C): Gaussian derivative filters of sigma = 1.4 on taps
// k = -kQualityRadius..kQualityRadius.
constexpr int kQualityRadius = 6;
struct QualityArgs {
    const void *Fe, *Fg, *A;                   // estimate, ground truth (w x h x 3), alpha_gt
    long long fe_pitch, fg_pitch, a_pitch;     // elements
    int w, h;
    float g[2 * kQualityRadius + 1];           // smoothing taps
    float dg[2 * kQualityRadius + 1];          // derivative taps
    double *partials;                          // 3 per block (quality_blocks)
};
long long quality_blocks(int w, int h);

// Sum of one double per thread over the block (blockDim.x a multiple of 32, at most
// 1024); `red` holds blockDim.x / 32 doubles. The result is valid in thread 0, and the
// order of the additions is fixed.
__device__ __forceinline__ double block_sum_d(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < nw) v = red[threadIdx.x];
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Converged reference (fg_minimiser_cg): preconditioned conjugate gradients in float64
// on grad E = 0. Vectors hold 6 n doubles: F (n x 3, row-major pixels) then B.
struct CgScalars {
    double rz, pq, alpha, beta, rr, bb;
};
struct CgArgs {
    const void *I, *A;
    long long I_pitch, A_pitch;   // elements
    int w, h;
    double eps, omega;
    double *x, *r, *z, *q;
    double *partials;             // 3 per block
    CgScalars *sc;                // device
};
int cg_blocks(int w, int h);
// r = b - H x, z = M^-1 r, p = z; rz, bb, rr; beta = 0.
cudaError_t cg_start(int dtype, const CgArgs &a, double *p, cudaStream_t s);
// One iteration: p_new = z + beta p_old, q = H p_new, alpha = rz / <p, q>, x += alpha p,
// r -= alpha q, z = M^-1 r, beta = <r, z> / rz, rr = <r, r>.
cudaError_t cg_iterate(int dtype, const CgArgs &a, const double *p_old, double *p_new,
                       cudaStream_t s);
// rr = |b - H x|^2 recomputed from x (into a.r, a.z used as scratch).
cudaError_t cg_true_residual(int dtype, const CgArgs &a, cudaStream_t s);
// SAD, MSE and GRAD into out[0..2] (device), via per-block partials.
cudaError_t launch_quality(int dtype, const QualityArgs &q, double *out, cudaStream_t s);

// Programmatic dependent launch. Kernels of a solve are launched so that the next one
// may be scheduled while the previous one drains: each kernel first waits for the grids
// it depends on to finish (and their memory to be visible), before its first global
// memory access of any kind; a block lets the dependents launch once its work is done.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_leave() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Lets `kernel` use dynamic shared memory up to the device's opt-in maximum less its
// static shared memory. The limit is always set to that largest value (never lowered), so
// every launch and every graph node captured for the kernel, whatever its own size, stays
// within the limit in force.
template <typename Kern>
cudaError_t allow_dynamic_smem(Kern *kernel) {
    int dev = 0, most = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&most, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                most - (int)fa.sharedSizeBytes);
}

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_level_pass(int dtype, int iters, int clamp, const PassArgs &a,
                              cudaStream_t s);
// Ring variant (TMA bulk row copies into a per-warp shared-memory ring): a.cap*/slot_bytes
// must be filled in; returns cudaErrorInvalidValue if iters is not 1 or 2.
cudaError_t launch_level_pass_ring(int dtype, int iters, int clamp, const PassArgs &a,
                                   cudaStream_t s);
size_t level_pass_ring_smem(int slot_bytes);

// Level pass with reflected borders and running sums (level_tile.cu): PassArgs tile_* and
// lt_* fields and the maps of the gathered images filled in; a.tile_slots (2 or 3) chunks
// in flight per warp. With blocks_per_sm != NULL it only reports the occupancy.
cudaError_t launch_level_tile(int dtype, int iters, int clamp, const PassArgs &a,
                              const TileMaps &m, cudaStream_t s, int *blocks_per_sm);
size_t level_tile_smem(int chunk_bytes, int slots);
// Work-list batch over level_tile strips (level_tile.cu): a pass's slots (BatchDesc
// a.tile_slots <= kBatchMaxSlots chunks of a.tile_chunk bytes) fill the warp's `region`
// bytes. With blocks_per_sm != NULL it only reports the occupancy.
constexpr int kBatchMaxSlots = 3;
size_t tile_batch_smem(int region);
cudaError_t launch_tile_batch(int dtype, int clamp, const BatchLaunch &b, cudaStream_t s,
                              int *blocks_per_sm);
// The tile pass's device error word (1 = a wait gave up), read and cleared; fg_sync reads
// it through read_and_clear_device_error.
cudaError_t read_and_clear_tile_error(int *code, cudaStream_t s);
// Small-level variant: one block per 32 x 16 output tile, all sweeps in shared memory.
// Red-black order: `iters` (1 or 2) red-black iterations of a level in one launch.
cudaError_t launch_level_rb(int dtype, int iters, int clamp, const PassArgs &a, cudaStream_t s);
// ---- cone kernel (cone.cu): a run of small levels in one launch.
// Each block owns a 32 x 16 tile of the run's last level and computes, in shared memory,
// every level of the run on the region its tile depends on (its dependency cone): the
// region a level's sweeps need, expanded by that level's sweep count, mapped down to the
// level below by the nearest-resize rule, back to the state the coarse kernel left.
constexpr int kConeMaxLevels = 8;
constexpr int kConeTW = 32, kConeTH = 16;

struct ConeRect {
    int x0, y0, x1, y1;   // inclusive
};

struct ConeArgs {
    const void *I;
    long long I_pitch;
    const void *A;
    long long A_pitch;
    int Iw, Ih;
    const void *Fs, *Bs;       // state of the level below the run (pitch s_pitch elements)
    long long s_pitch;
    int sw, sh;
    void *Fd, *Bd;             // state of the run's last level
    long long d_pitch;
    float eps, omega;
    int nlev;
    int lw[kConeMaxLevels], lh[kConeMaxLevels], lk[kConeMaxLevels];
    int cap;                   // cells of the largest region of any block (shared-memory sizing)
    int io;                    // cells of all the run's regions of a block together, at most
    const void *Bn;            // compositing epilogue (run ending at the top level), as PassArgs
    void *In;
    long long bn_pitch, in_pitch;
};

// The regions of block (bx, by): E[l] = the cells of level l its sweeps start from, and
// *Rc = the cells of the level below the run that the first level's start reads.
__host__ __device__ inline int cone_lo(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int cone_hi(int a, int b) { return a > b ? a : b; }

__host__ __device__ inline void cone_regions(const ConeArgs &a, int bx, int by, ConeRect *E,
                                             ConeRect *Rc) {
    const int L = a.nlev - 1;
    ConeRect R{bx * kConeTW, by * kConeTH, cone_lo(bx * kConeTW + kConeTW - 1, a.lw[L] - 1),
               cone_lo(by * kConeTH + kConeTH - 1, a.lh[L] - 1)};
    for (int l = L; l >= 0; --l) {
        const int w = a.lw[l], h = a.lh[l], k = a.lk[l];
        const ConeRect e{cone_hi(R.x0 - k, 0), cone_hi(R.y0 - k, 0), cone_lo(R.x1 + k, w - 1),
                         cone_lo(R.y1 + k, h - 1)};
        E[l] = e;
        const int pw = l > 0 ? a.lw[l - 1] : a.sw, ph = l > 0 ? a.lh[l - 1] : a.sh;
        R = ConeRect{nearest_src(e.x0, pw, w), nearest_src(e.y0, ph, h), nearest_src(e.x1, pw, w),
                     nearest_src(e.y1, ph, h)};
    }
    *Rc = R;
}

cudaError_t launch_cone(int dtype, int clamp, const ConeArgs &a, cudaStream_t s);
size_t cone_smem_bytes(int cap, int io);

cudaError_t launch_level_small(int dtype, int iters, int clamp, const PassArgs &a,
                               cudaStream_t s);
int level_pass_tile_rows();
// Device error word of the library's bounded waits (0 = no error).
cudaError_t read_and_clear_device_error(int *code, cudaStream_t s);
// Enqueues on s copies of the two device error words into dst[0] and dst[1] (host memory,
// pinned for the copy to stay asynchronous), without clearing them.
cudaError_t enqueue_device_error_read(int *dst, cudaStream_t s);
cudaError_t enqueue_tile_error_read(int *dst, cudaStream_t s);
cudaError_t launch_coarse(int dtype, int clamp, const CoarseArgs &a, cudaStream_t s);
// Coarse levels of many images, one block per image (list: device array of n args).
cudaError_t launch_coarse_batch(int dtype, int clamp, const CoarseArgs *list, int n,
                                int max_total, cudaStream_t s);
size_t coarse_smem_bytes(int total_pixels);

}  // namespace fgml
