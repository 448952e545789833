// Device helpers of the strip kernels (level_tile.cu): packed float32x2 arithmetic, index
// reflection, shared-memory loads of the storage types, the edge weight and the 2x2
// inverse of the per-pixel solve (Section III-C), async copies and the chunk mbarriers.
// Included inside the file's anonymous namespace.
#pragma once

constexpr unsigned kMask = 0xffffffffu;
constexpr int kW = 60;             // output columns per warp
constexpr int kWarps = 4;          // warps per block
constexpr int kChunkRows = 4;      // rows per TMA gather (gather4)
constexpr int kPolls = 1 << 20;    // try_wait polls before a wait gives up
constexpr uint32_t kHintNs = 2000; // suspend-time hint of one poll
#ifndef FGML_TILE_BLOCKS
#define FGML_TILE_BLOCKS 3
#endif

using f2 = float2;
__device__ __forceinline__ f2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Index v reflected into [0, n): -1 -> 0, -2 -> 1, n -> n - 1, n + 1 -> n - 2, clamped.
__device__ __forceinline__ int reflect(int v, int n) {
    if (v < 0) v = -1 - v;
    if (v >= n) v = 2 * n - 1 - v;
    return min(max(v, 0), n - 1);
}

// ------------------------------------------------------------------ loads and stores

template <typename T> __device__ __forceinline__ float ldsh(const unsigned char *p);
template <> __device__ __forceinline__ float ldsh<float>(const unsigned char *p) {
    return *reinterpret_cast<const float *>(p);
}
template <> __device__ __forceinline__ float ldsh<__nv_bfloat16>(const unsigned char *p) {
    return __uint_as_float((uint32_t)*reinterpret_cast<const unsigned short *>(p) << 16);
}
template <> __device__ __forceinline__ float ldsh<__half>(const unsigned char *p) {
    return __half2float(*reinterpret_cast<const __half *>(p));
}

// The two 16-bit values of a 32-bit word as floats (low half first).
__device__ __forceinline__ f2 unpack(uint32_t w, const __nv_bfloat16 *) {
    return mk(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ f2 unpack(uint32_t w, const __half *) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}

__device__ __forceinline__ void st_pair(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void st_pair(__half *p, float a, float b) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void st_pair(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}


__device__ __forceinline__ float edge(float ai, float aj, float eps, float omega) {
    return fmaf(omega, fabsf(ai - aj), eps);
}


// Inverse of A = [[a^2 + S, a(1-a)], [a(1-a), (1-a)^2 + S]] as (mFF, mBB, mFB) with
// A^{-1} = [[mFF, -mFB], [-mFB, mBB]].
__device__ __forceinline__ void invert(f2 a, f2 S, f2 &mFF, f2 &mBB, f2 &mFB) {
    const f2 be = mk(1.f - a.x, 1.f - a.y);
    const f2 A00 = fma2(a, a, S);
    const f2 A11 = fma2(be, be, S);
    const f2 A01 = mul2(a, be);
    const f2 pd = mul2(A00, A11);
    const float d0 = fmaf(-A01.x, A01.x, pd.x), d1 = fmaf(-A01.y, A01.y, pd.y);
    const f2 m = mk(__fdividef(1.f, d0), __fdividef(1.f, d1));
    mFF = mul2(A11, m);
    mBB = mul2(A00, m);
    mFB = mul2(A01, m);
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
}

// The calling warp's chunk mbarriers: `n` of them at bar0, initialised once (arrival
// count 1: lane 0's arrival that also sets the bytes the gathers deliver) and used by
// every strip the warp runs; per-lane copies add their own arrivals before lane 0's.
__device__ __forceinline__ void init_chunk_barriers(uint32_t bar0, int n) {
    if ((threadIdx.x & 31) == 0) {
        for (int s = 0; s < n; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0 + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}
