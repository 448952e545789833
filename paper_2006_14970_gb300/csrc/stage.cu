// Row-aligned copies of input images. Tensor maps need every row to start on the 16-byte
// grid; an image whose rows do not (a tightly packed width that is not a multiple of 16
// bytes) is copied once into a buffer whose pitch is rounded up to 16 bytes, so that its
// level passes can take the TMA tile path instead of per-row copies. One launch copies
// any number of images: blocks stride over the rows of all jobs together (so big images
// get blocks in proportion), threads walk a row's 16-byte chunks, each written from
// element-sized loads of the source row.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) stage_rows_kernel(const StageList list, int njobs,
                                                              long long total_rows) {
    pdl_enter();
    constexpr int kPer = 16 / sizeof(T);
    constexpr int kUnroll = 4;   // chunks per thread per round: their loads all issue first
    // blocks stride over the rows of all jobs together (jobs hold their first global row)
    for (long long g = blockIdx.x; g < total_rows; g += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {   // last job whose first row is <= g
            const int mid = (lo + hi + 1) / 2;
            const long long r0 = list.dev ? list.dev[mid].row0 : list.local[mid].row0;
            if (r0 <= g) lo = mid;
            else hi = mid - 1;
        }
        const StageJob &j = list.dev ? list.dev[lo] : list.local[lo];
        const long long r = g - j.row0;
        const int chunks = (int)((j.row_bytes + 15) / 16);
        const int row_elems = (int)(j.row_bytes / (long long)sizeof(T));
        const T *src = reinterpret_cast<const T *>(static_cast<const char *>(j.src) + r * j.src_pitch);
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<char *>(j.dst) + r * j.dst_pitch);
        for (int c0 = threadIdx.x; c0 < chunks; c0 += kThreads * kUnroll) {
            union Chunk {
                uint4 v;
                T e[kPer];
            } u[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int c = c0 + q * kThreads;
                u[q].v = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int k = 0; k < kPer; ++k)
                    if (c * kPer + k < row_elems) u[q].e[k] = __ldg(src + c * kPer + k);
            }
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int c = c0 + q * kThreads;
                if (c < chunks) dst[c] = u[q].v;
            }
        }
    }
    pdl_leave();
}

}  // namespace

cudaError_t launch_stage_rows(int dtype, const StageList &list, int njobs, long long total_rows,
                              cudaStream_t s) {
    if (njobs < 1 || total_rows < 1 || (!list.dev && njobs > 2)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(total_rows, 152 * 8);
    switch (dtype) {
        case kF32: return launch_pdl(stage_rows_kernel<float>, dim3(grid), dim3(kThreads), 0, s, list, njobs, total_rows);
        case kBF16:
            return launch_pdl(stage_rows_kernel<__nv_bfloat16>, dim3(grid), dim3(kThreads), 0, s, list, njobs,
                              total_rows);
        case kF16: return launch_pdl(stage_rows_kernel<__half>, dim3(grid), dim3(kThreads), 0, s, list, njobs, total_rows);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml

namespace fgml {
namespace {

// Counts the values of a w x h x ch image outside [0, 1] (NaN included) into *bad.
template <typename T>
__global__ void __launch_bounds__(256) range_check_kernel(const T *p, long long pitch, int w, int h,
                                                          int ch, unsigned long long *bad) {
    const long long row = (long long)w * ch;
    unsigned long long mine = 0;
    for (long long y = blockIdx.x; y < h; y += gridDim.x)
        for (long long x = threadIdx.x; x < row; x += blockDim.x) {
            const float v = ld_elem(p + y * pitch + x);
            if (!(v >= 0.f && v <= 1.f)) ++mine;
        }
    if (mine) atomicAdd(bad, mine);
}

}  // namespace

cudaError_t launch_range_check(int dtype, const void *p, long long pitch, int w, int h, int ch,
                               unsigned long long *bad, cudaStream_t s) {
    const int grid = std::max(1, std::min(h, 1216));
    switch (dtype) {
        case kF32: range_check_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(p), pitch, w, h, ch, bad); break;
        case kBF16:
            range_check_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(p), pitch, w, h, ch, bad);
            break;
        case kF16: range_check_kernel<__half><<<grid, 256, 0, s>>>(static_cast<const __half *>(p), pitch, w, h, ch, bad); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fgml
