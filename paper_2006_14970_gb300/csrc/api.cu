// Host side of libfgml: argument checks, the level planner, per-stream workspaces and
// the launch sequence of the multi-level method (Algorithm 1).
#include "fgml.h"
#include "fgml_internal.h"
#include "serve_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <utility>
#include <vector>

namespace fgml {
int level_pass_strip_width();
int level_pass_warps_per_block();
}

namespace {

using namespace fgml;

thread_local std::string g_err;

fg_status fail(fg_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

fg_status cuda_fail(cudaError_t e, const char *what) {
    return fail(FG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kMaxSide = 32767;

int elem_size(fg_dtype d) { return d == FG_F32 ? 4 : 2; }

// ------------------------------------------------------------------ level planner

// n_l = ceil(log2(max(w, h))), at least 1 (Algorithm 1).
int level_count(int w, int h) {
    const unsigned m = (unsigned)std::max(w, h);
    const int n = m <= 1 ? 0 : 32 - __builtin_clz(m - 1u);
    return std::max(n, 1);
}

// round(side^(l/n)), rounding halves up (exact halves cannot occur).
int level_side(int side, int l, int n) {
    return (int)std::lround(std::pow((double)side, (double)l / (double)n));
}

struct Level {
    int w, h, k;
};

// Levels 1..nc run in the one-block coarse kernel: the longest prefix of levels with at
// most kCoarseCap pixels each and kCoarseTotal together (level 1 is at most 2 x 2).
int coarse_levels(const std::vector<Level> &lv) {
    int nc = 0;
    long long total = 0;
    while (nc < (int)lv.size() && nc < kCoarseMaxLevels) {
        const long long n = (long long)lv[nc].w * lv[nc].h;
        if (n > kCoarseCap || total + n > kCoarseTotal) break;
        total += n;
        ++nc;
    }
    return nc;
}

std::vector<Level> plan_levels(int w, int h, const fg_params &p) {
    const int n = level_count(w, h);
    std::vector<Level> lv(n);
    for (int l = 1; l <= n; ++l) {
        Level &L = lv[l - 1];
        L.w = level_side(w, l, n);
        L.h = level_side(h, l, n);
        L.k = (L.w <= p.small_size && L.h <= p.small_size) ? p.small_iters : p.big_iters;
    }
    return lv;
}

// ------------------------------------------------------------------ checks

fg_status check_params(const fg_params &p) {
    if (!(p.eps_r > 0.f) || !std::isfinite(p.eps_r))
        return fail(FG_ERR_INVALID_ARG, "eps_r must be finite and > 0");
    if (!(p.omega >= 0.f) || !std::isfinite(p.omega))
        return fail(FG_ERR_INVALID_ARG, "omega must be finite and >= 0");
    if (p.small_iters < 0 || p.big_iters < 0 || p.small_size < 0)
        return fail(FG_ERR_INVALID_ARG, "iteration counts and small_size must be >= 0");
    if (p.small_iters > 1000000 || p.big_iters > 1000000)
        return fail(FG_ERR_INVALID_ARG, "iteration counts above 1e6");
    if (p.order != FG_ORDER_JACOBI && p.order != FG_ORDER_REDBLACK)
        return fail(FG_ERR_UNSUPPORTED, "order %d is not available on the GPU (Jacobi or red-black)", p.order);
    if (!std::isfinite(p.init)) return fail(FG_ERR_INVALID_ARG, "init must be finite");
    return FG_OK;
}

fg_status check_image(const fg_image *im, int ch, const char *name) {
    if (!im) return fail(FG_ERR_INVALID_ARG, "%s is NULL", name);
    if (!im->ptr) return fail(FG_ERR_INVALID_ARG, "%s->ptr is NULL", name);
    if (im->w < 1 || im->h < 1 || im->w > kMaxSide || im->h > kMaxSide)
        return fail(FG_ERR_INVALID_ARG, "%s size %dx%d outside [1, %d]", name, im->w, im->h,
                    kMaxSide);
    if (im->dtype != FG_F32 && im->dtype != FG_BF16 && im->dtype != FG_F16)
        return fail(FG_ERR_INVALID_ARG, "%s has an unknown dtype %d", name, (int)im->dtype);
    const int es = elem_size(im->dtype);
    if (im->row_pitch_bytes < (long long)im->w * ch * es || im->row_pitch_bytes % es)
        return fail(FG_ERR_INVALID_ARG, "%s row pitch %lld invalid for width %d", name,
                    im->row_pitch_bytes, im->w);
    if (((uintptr_t)im->ptr) % es) return fail(FG_ERR_INVALID_ARG, "%s is misaligned", name);
    return FG_OK;
}

// byte range [lo, hi) an image spans
std::pair<uintptr_t, uintptr_t> span(const fg_image *im, int ch) {
    const uintptr_t lo = (uintptr_t)im->ptr;
    const uintptr_t hi = lo + (uintptr_t)(im->row_pitch_bytes * (im->h - 1)) +
                         (uintptr_t)im->w * ch * elem_size(im->dtype);
    return {lo, hi};
}

bool overlap(const fg_image *a, int ca, const fg_image *b, int cb) {
    auto x = span(a, ca), y = span(b, cb);
    return x.first < y.second && y.first < x.second;
}

// NVTX range over one entry point (shows in profilers' timelines; a no-op without a tool).
struct Range {
    explicit Range(const char *m) { nvtxRangePushA(m); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ------------------------------------------------------------------ workspaces

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Workspace {
    Buf lev[2];   // intermediate level states: F then B, each w x h x 3
    Buf stage;    // device staging of the host-memory entry point
    Buf batch;    // per-image levels (and row-aligned copies) of fg_estimate_batch
    Buf worklist; // device copy of the last directly launched work list
    Buf aux;      // per-block partial sums of fg_quality
    Buf cg;       // vectors of fg_minimiser_cg
    Buf check;    // counter of the optional input range check
    Buf align;    // copies of I and alpha with rows on the 16-byte grid (tensor maps need it)
    // launch sequences of fg_estimate captured as CUDA graphs, by call signature
    std::map<std::string, cudaGraphExec_t> graphs;
    std::vector<std::string> graph_order;   // oldest first, for eviction
    // work lists owned by cached batch graphs (each graph reads its own copy)
    std::map<std::string, Buf> graph_bufs;
    // batch signatures seen once: a batch is captured when it comes a second time, so
    // one-off batches (a server's) never pay for a capture
    std::vector<std::string> batch_seen;
};

constexpr size_t kMaxGraphs = 64;   // cached launch graphs per workspace

// The workspace of stream s drops its cached graphs; the work lists they own are freed in
// stream order, after the launches already queued on s.
void clear_graphs(Workspace &ws, cudaStream_t s) {
    for (auto &kv : ws.graphs) cudaGraphExecDestroy(kv.second);
    ws.graphs.clear();
    ws.graph_order.clear();
    for (auto &kv : ws.graph_bufs) cudaFreeAsync(kv.second.p, s);
    ws.graph_bufs.clear();
}

// Drops the oldest cached graph (and the work list it owns) once the cache is full.
void evict_graphs(Workspace &ws, cudaStream_t s) {
    while (ws.graphs.size() >= kMaxGraphs) {
        const std::string k = ws.graph_order.front();
        cudaGraphExecDestroy(ws.graphs[k]);
        ws.graphs.erase(k);
        ws.graph_order.erase(ws.graph_order.begin());
        auto b = ws.graph_bufs.find(k);
        if (b != ws.graph_bufs.end()) {
            cudaFreeAsync(b->second.p, s);
            ws.graph_bufs.erase(b);
        }
    }
}

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

Workspace &workspace_for(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    return g_ws[{current_device(), s}];
}

fg_status ensure(Buf &b, size_t need, cudaStream_t s) {
    if (b.bytes >= need) return FG_OK;
    // host-side fault injection for tests: FGML_FAIL_ALLOC=1 refuses workspace growth
    if (const char *f = std::getenv("FGML_FAIL_ALLOC"))
        if (*f && *f != '0') return fail(FG_ERR_OOM, "workspace allocation of %zu bytes refused (FGML_FAIL_ALLOC)", need);
    if (b.p) {
        cudaStreamSynchronize(s);   // the old buffer may still be read by queued work
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(FG_ERR_OOM, "workspace allocation of %zu bytes failed: %s", need,
                    cudaGetErrorString(e));
    }
    b.bytes = need;
    return FG_OK;
}

int sm_count() {
    static int cache[64] = {0};
    const int d = current_device();
    if (d < 0 || d >= 64) return 148;
    if (!cache[d]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        cache[d] = v > 0 ? v : 148;
    }
    return cache[d];
}

// A level state (F and B) stored inside a workspace buffer.
struct State {
    const void *F, *B;
    long long pitch;   // elements
    int w, h;
    bool padded;       // rows are padded to 16 bytes inside the allocation (workspace)
};

// Rows of a workspace state are padded to 16 bytes so that tensor copies can read them.
long long state_pitch(int w, int es) {
    const long long q = 16 / es;
    return (3LL * w + q - 1) / q * q;
}

size_t state_bytes(int w, int h, int es) {
    const size_t plane = ((size_t)state_pitch(w, es) * h * es + 255) & ~(size_t)255;
    return 2 * plane;
}

State state_in(const Buf &b, int w, int h, int es) {
    const size_t plane = ((size_t)state_pitch(w, es) * h * es + 255) & ~(size_t)255;
    State s;
    s.F = b.p;
    s.B = (const char *)b.p + plane;
    s.pitch = state_pitch(w, es);
    s.w = w;
    s.h = h;
    s.padded = true;
    return s;
}

// ------------------------------------------------------------------ launches

struct Input {
    const void *I, *A;
    long long I_pitch, A_pitch;   // elements
    int w, h;
    bool padded = false;          // rows readable up to the pitch (the library's aligned copies)
};

// Rows per warp of a level pass: one wave of resident warps (two 4-warp blocks per SM)
// when the level is wide enough, so that every warp walks one tall strip and the
// vertical halo (2 rows above and below each strip) stays a small fraction.
int strip_rows(int w, int h, int blocks_per_sm = 2) {
    const int nx = (w + level_pass_strip_width() - 1) / level_pass_strip_width();
    const long long resident = (long long)sm_count() * blocks_per_sm * level_pass_warps_per_block();
    const long long ny = std::max<long long>(1, resident / nx);
    long long r = (h + ny - 1) / ny;
    return (int)std::max<long long>(r, 1);
}

// FGML_CONE=0 runs the small levels of a solve one launch each (for comparison).
bool cone_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("FGML_CONE");
        return !(e && *e == '0');
    }();
    return on;
}

// Levels up to this many pixels run in the small-level kernel (latency bound);
// FGML_SMALL_LEVEL_PIXELS overrides it for tuning.
long long small_level_pixels() {
    static const long long v = [] {
        const char *e = std::getenv("FGML_SMALL_LEVEL_PIXELS");
        return e && *e ? std::atoll(e) : 300000LL;
    }();
    return v;
}

// Shared memory of one ring-variant block; two blocks must fit on an SM.
constexpr size_t kRingSmemBudget = 110 * 1024;

// ------------------------------------------------------------------ tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        cudaGetLastError();
    });
    return fn;
}

// A 2D tensor map of `rows` rows of `inner8` 8-byte elements, `pitch` bytes apart, with
// a one-row box of `box8` elements (for gather-mode copies); false if the layout does
// not allow tensor copies (base or pitch off the 16-byte grid, box too wide).
// A tensor map over `rows` rows of `inner` elements of `unit` bytes (8, 4 or 2: the
// element type only sets the addressing granularity), boxes of `box` x 1 elements.
bool make_map(CUtensorMap *m, const void *base, long long inner, long long rows, long long pitch,
              int box, int unit) {
    EncodeTiledFn fn = encode_tiled();
    const CUtensorMapDataType ty = unit == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                 : unit == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                             : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    if (!fn || (unit != 8 && unit != 4 && unit != 2) || (reinterpret_cast<uintptr_t>(base) & 15) ||
        (pitch & 15) || box > 256 || box < 1 || (box * unit) % 16 || inner < 1 || inner * unit > pitch)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t boxd[2] = {(cuuint32_t)box, 1};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, ty, 2, const_cast<void *>(base), dims, strides, boxd, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Element unit, box width and row length (in units) for a tensor whose rows hold
// `rowbytes` bytes and whose strips span `span` bytes: the largest unit (8, 4, 2) that
// divides the row (or, for a padded state, whose rounded-up row stays inside the pitch)
// and gives a box of at most 256 elements.
bool pick_unit(long long rowbytes, int span, bool padded, long long pitch, int &unit, int &box,
               long long &inner) {
    for (int u : {8, 4, 2}) {
        const int g = 16 / u;
        const int b = ((15 + span + u - 1) / u + g - 1) / g * g;
        if (b > 256) continue;
        if (rowbytes % u == 0) {
            inner = rowbytes / u;
        } else if (padded && (rowbytes + u - 1) / u * u <= pitch) {
            inner = (rowbytes + u - 1) / u;
        } else {
            continue;
        }
        unit = u;
        box = b;
        return true;
    }
    return false;
}

// Chunk layout of a level_tile pass: each image is gathered through a tensor map where
// its layout allows one and the strip's source span fits one box, and is otherwise copied
// by the lanes (their own pixels only). False if a 16-bit image would need per-lane copies
// but its base or row pitch is off the 4-byte grid (4-byte copies would then straddle).
// With max_chunk > 0, I and alpha are copied by the lanes whenever gathering them would
// make a chunk slot larger than max_chunk bytes (the work-list batch keeps its per-warp
// region small enough for two blocks per SM).
bool plan_chunks(int dtype, const Input &in, const State &src, PassArgs &a, TileMaps &m,
                 int max_chunk = 0) {
    const int es = dtype == kF32 ? 4 : 2;
    auto r128 = [](int v) { return (v + 127) & ~127; };
    const int R = level_pass_tile_rows();
    const int spanI = strip_span(in.w, a.w), spanS = strip_span(src.w, a.w);
    const long long rbI = 3LL * in.w * es, rbA = (long long)in.w * es, rbS = 3LL * src.w * es;
    long long inI = 0, inA = 0, inS = 0;
    bool fitI = true;
    if (max_chunk > 0) {
        // a chunk with I and alpha gathered and F and B gathered or copied (upper bound)
        const int lane_px = es == 4 ? 24 : 16;
        const int boxI = 3 * spanI * es + 32, boxA = spanI * es + 32;
        const int boxS = std::max(3 * spanS * es + 32, 32 * lane_px);
        fitI = r128(R * boxI) + r128(R * boxA) + 2 * r128(R * boxS) <= max_chunk;
    }
    const bool tI = fitI && pick_unit(rbI, 3 * spanI * es, in.padded, in.I_pitch * es, a.tile_uI, a.tile_bwI, inI) &&
                    make_map(&m.I, in.I, inI, in.h, in.I_pitch * es, a.tile_bwI, a.tile_uI);
    const bool tA = fitI && pick_unit(rbA, spanI * es, in.padded, in.A_pitch * es, a.tile_uA, a.tile_bwA, inA) &&
                    make_map(&m.A, in.A, inA, in.h, in.A_pitch * es, a.tile_bwA, a.tile_uA);
    const bool tS = pick_unit(rbS, 3 * spanS * es, src.padded, src.pitch * es, a.tile_uS, a.tile_bwS, inS) &&
                    make_map(&m.F, src.F, inS, src.h, src.pitch * es, a.tile_bwS, a.tile_uS) &&
                    make_map(&m.B, src.B, inS, src.h, src.pitch * es, a.tile_bwS, a.tile_uS);
    auto words_ok = [&](const void *base, long long pitch_bytes) {
        return es == 4 || (((uintptr_t)base & 3) == 0 && (pitch_bytes & 3) == 0);
    };
    if ((!tI && !words_ok(in.I, in.I_pitch * es)) || (!tA && !words_ok(in.A, in.A_pitch * es)) ||
        (!tS && !(words_ok(src.F, src.pitch * es) && words_ok(src.B, src.pitch * es))))
        return false;
    // images copied by the lanes keep valid (unused) box units for the kernel's set-up
    if (!tI) a.tile_uI = 8;
    if (!tA) a.tile_uA = 8;
    if (!tS) a.tile_uS = 8;
    a.lt_mode[0] = !tI;
    a.lt_mode[1] = !tA;
    a.lt_mode[2] = a.lt_mode[3] = !tS;
    const int lane_px = es == 4 ? 24 : 16;   // bytes per lane of a 3-channel image (two pixels)
    a.lt_row[0] = tI ? a.tile_bwI * a.tile_uI : 32 * lane_px;
    a.lt_row[1] = tA ? a.tile_bwA * a.tile_uA : 32 * 8;
    a.lt_row[2] = a.lt_row[3] = tS ? a.tile_bwS * a.tile_uS : 32 * lane_px;
    a.lt_off[0] = 0;
    for (int k = 0; k < 3; ++k) a.lt_off[k + 1] = a.lt_off[k] + r128(R * a.lt_row[k]);
    a.tile_chunk = a.lt_off[3] + r128(R * a.lt_row[3]);
    a.tile_tx = R * ((tI ? a.lt_row[0] : 0) + (tA ? a.lt_row[1] : 0) + (tS ? 2 * a.lt_row[2] : 0));
    return true;
}

// Compositing epilogue of the last pass of a solve (fg_estimate_composite).
struct Composite {
    const void *Bn = nullptr;
    void *In = nullptr;
    long long bn_pitch = 0, in_pitch = 0;   // elements
};

cudaError_t pass(int dtype, int iters, int clamp, const fg_params &p, const Input &in,
                 const State &src, void *Fd, void *Bd, long long d_pitch, int w, int h,
                 cudaStream_t s, const Composite *cmp = nullptr) {
    PassArgs a;
    std::memset(&a, 0, sizeof a);
    if (cmp) {
        a.Bn = cmp->Bn;
        a.In = cmp->In;
        a.bn_pitch = cmp->bn_pitch;
        a.in_pitch = cmp->in_pitch;
    }
    a.I = in.I;
    a.I_pitch = in.I_pitch;
    a.A = in.A;
    a.A_pitch = in.A_pitch;
    a.Iw = in.w;
    a.Ih = in.h;
    a.Fs = src.F;
    a.Bs = src.B;
    a.s_pitch = src.pitch;
    a.sw = src.w;
    a.sh = src.h;
    a.Fd = Fd;
    a.Bd = Bd;
    a.d_pitch = d_pitch;
    a.w = w;
    a.h = h;
    a.eps = p.eps_r;
    a.omega = p.omega;
    a.strip_h = strip_rows(w, h);
    a.n_xstrips = (w + level_pass_strip_width() - 1) / level_pass_strip_width();
    a.n_warps = a.n_xstrips * ((h + a.strip_h - 1) / a.strip_h);
    a.capI = a.capA = a.capS = a.slot_bytes = 0;
    if (p.order == FG_ORDER_REDBLACK && (iters == 1 || iters == 2))
        return launch_level_rb(dtype, iters, clamp, a, s);
    if ((iters == 1 || iters == 2) && (long long)w * h <= small_level_pixels())
        return launch_level_small(dtype, iters, clamp, a, s);
    if (iters == 1 || iters == 2) {
        TileMaps maps;
        if (plan_chunks(dtype, in, src, a, maps)) {
            // the most resident warps, then the most chunks in flight
            int best_occ = 0, best_slots = 0;
            for (int sl : {3, 2}) {
                a.tile_slots = sl;
                int occ = 0;
                if (launch_level_tile(dtype, iters, clamp, a, maps, s, &occ) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                if (occ > best_occ) {
                    best_occ = occ;
                    best_slots = sl;
                }
            }
            if (best_occ > 0) {
                a.tile_slots = best_slots;
                a.strip_h = strip_rows(w, h, best_occ);
                a.n_warps = a.n_xstrips * ((h + a.strip_h - 1) / a.strip_h);
                return launch_level_tile(dtype, iters, clamp, a, maps, s, nullptr);
            }
        }
        // 16-bit rows off the 4-byte grid whose levels cannot be gathered through tensor
        // maps: the row-ring or plain-load kernels
        // ring slots: each segment's 16-byte aligned superset (up to 30 extra bytes)
        const int es = dtype == kF32 ? 4 : 2;
        auto r16 = [](int v) { return (v + 15) & ~15; };
        const int spanI = strip_span(in.w, w), spanS = strip_span(src.w, w);
        a.capI = r16(3 * spanI * es + 30);
        a.capA = r16(spanI * es + 30);
        a.capS = r16(3 * spanS * es + 30);
        a.slot_bytes = a.capI + a.capA + 2 * a.capS;
        a.I_end = (const char *)in.I + ((long long)(in.h - 1) * in.I_pitch + 3LL * in.w) * es;
        a.A_end = (const char *)in.A + ((long long)(in.h - 1) * in.A_pitch + in.w) * es;
        a.Fs_end = (const char *)src.F + ((long long)(src.h - 1) * src.pitch + 3LL * src.w) * es;
        a.Bs_end = (const char *)src.B + ((long long)(src.h - 1) * src.pitch + 3LL * src.w) * es;
        if (level_pass_ring_smem(a.slot_bytes) <= kRingSmemBudget)
            return launch_level_pass_ring(dtype, iters, clamp, a, s);
    }
    return launch_level_pass(dtype, iters, clamp, a, s);
}

// Sweep counts of the passes of a level with k sweeps: at most 2 per pass.
std::vector<int> split_sweeps(int k) {
    std::vector<int> v;
    if (k == 0) {
        v.push_back(0);
        return v;
    }
    if (k % 2) v.push_back(1);
    for (int i = 0; i < k / 2; ++i) v.push_back(2);
    return v;
}

// Runs the passes of one level from `src` (in workspace buffer *buf, or -1 for caller
// memory). Every pass reads one buffer and writes the other; the last pass writes to
// (Fd, Bd) when `to_caller`, else to a workspace buffer. On return src/buf describe the
// level's final state when it stays in the workspace.
fg_status run_level(int dtype, const fg_params &p, const Input &in, State &src, int &buf,
                    int k, int w, int h, bool to_caller, void *Fd, void *Bd, long long d_pitch,
                    Workspace &ws, int es, cudaStream_t s, const Composite *cmp = nullptr) {
    const std::vector<int> passes = split_sweeps(k);
    for (size_t j = 0; j < passes.size(); ++j) {
        if (to_caller && j + 1 == passes.size()) {
            cudaError_t e = pass(dtype, passes[j], p.clamp, p, in, src, Fd, Bd, d_pitch, w, h, s, cmp);
            if (e != cudaSuccess) return cuda_fail(e, "level pass launch");
        } else {
            const int nb = buf == 0 ? 1 : 0;
            State dst = state_in(ws.lev[nb], w, h, es);
            cudaError_t e = pass(dtype, passes[j], p.clamp, p, in, src, (void *)dst.F,
                                 (void *)dst.B, dst.pitch, w, h, s);
            if (e != cudaSuccess) return cuda_fail(e, "level pass launch");
            src = dst;
            buf = nb;
        }
    }
    return FG_OK;
}

// Rows a tensor map can describe: base and pitch (bytes) on the 16-byte grid.
bool rows_on_grid(const void *ptr, long long pitch_bytes) {
    return ((uintptr_t)ptr & 15) == 0 && (pitch_bytes & 15) == 0;
}

// Whether a solve reads a row-aligned copy of its input (rows off the 16-byte grid), or
// its level passes read the input in place by per-lane 4-byte copies. Measured: float32
// images up to 8 Mpx are faster read in place (the 64-image batch 1.10 vs 1.17 ms, 1001x777
// 64.6 vs 68.7 us), larger ones and 16-bit storage faster staged (the batch in bfloat16
// 1.34 vs 1.43 ms); 16-bit rows off the 4-byte grid must be staged. FGML_STAGE=1 stages
// every off-grid input, FGML_STAGE=0 none that can be read in place.
bool needs_stage(const Input &in, int es) {
    if (rows_on_grid(in.I, in.I_pitch * es) && rows_on_grid(in.A, in.A_pitch * es)) return false;
    static const int mode = [] {
        const char *e = std::getenv("FGML_STAGE");
        return e && *e == '0' ? 0 : e && *e == '1' ? 1 : 2;
    }();
    auto words = [&](const void *p, long long pitch_bytes) {
        return ((uintptr_t)p & 3) == 0 && (pitch_bytes & 3) == 0;
    };
    if (es == 2 && !(words(in.I, in.I_pitch * es) && words(in.A, in.A_pitch * es))) return true;
    if (mode != 2) return mode == 1;
    return es == 2 || (long long)in.w * in.h > (8LL << 20);
}

// Last level of the run of small levels above the coarse ones that one cone launch
// computes: consecutive levels of at most small_level_pixels() each (at most
// kConeMaxLevels of them), Jacobi order only; nc - 1 when there is none.
int cone_run(const std::vector<Level> &lv, int nc, const fg_params &p) {
    int m = nc - 1;
    if (p.order != FG_ORDER_JACOBI || nc < 1 || !cone_enabled()) return m;
    while (m + 1 < (int)lv.size() && m + 1 - nc < kConeMaxLevels &&
           (long long)lv[m + 1].w * lv[m + 1].h <= small_level_pixels())
        ++m;
    return m;
}

// Arguments of the cone launch for levels nc..m, reading the coarse kernel's output
// `src`; false when the largest region of a block would need more than kConeSmemMax bytes
// of shared memory (many sweeps per level), and the levels then run one launch each.
constexpr size_t kConeSmemMax = 100 * 1024;
bool plan_cone(const Input &in, const std::vector<Level> &lv, int nc, int m, const State &src,
               const fg_params &p, ConeArgs &a) {
    std::memset(&a, 0, sizeof a);
    a.I = in.I;
    a.I_pitch = in.I_pitch;
    a.A = in.A;
    a.A_pitch = in.A_pitch;
    a.Iw = in.w;
    a.Ih = in.h;
    a.Fs = src.F;
    a.Bs = src.B;
    a.s_pitch = src.pitch;
    a.sw = src.w;
    a.sh = src.h;
    a.eps = p.eps_r;
    a.omega = p.omega;
    a.nlev = m - nc + 1;
    for (int i = 0; i < a.nlev; ++i) {
        a.lw[i] = lv[nc + i].w;
        a.lh[i] = lv[nc + i].h;
        a.lk[i] = lv[nc + i].k;
    }
    // the largest region over the blocks (edge blocks are clipped, interior ones alike)
    const int gx = (a.lw[a.nlev - 1] + kConeTW - 1) / kConeTW, gy = (a.lh[a.nlev - 1] + kConeTH - 1) / kConeTH;
    long long cap = 0, io = 0;
    ConeRect E[kConeMaxLevels], Rc;
    auto cells = [](const ConeRect &r) { return (long long)(r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1); };
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
            cone_regions(a, bx, by, E, &Rc);
            cap = std::max(cap, cells(Rc));
            long long sum = 0;
            for (int i = 0; i < a.nlev; ++i) {
                cap = std::max(cap, cells(E[i]));
                sum += cells(E[i]);
            }
            io = std::max(io, sum);
        }
    if (cone_smem_bytes((int)std::min<long long>(cap, 1 << 20), (int)std::min<long long>(io, 1 << 20)) >
        kConeSmemMax)
        return false;
    a.cap = (int)cap;
    a.io = (int)io;
    return true;
}

// The kernels of one solve, enqueued on `s` (no allocation, no synchronisation).
fg_status launch_sequence(const Input &in, int dtype, const fg_params &p,
                          const std::vector<Level> &lv, int nc, void *Fd, void *Bd,
                          long long d_pitch, Workspace &ws, int es, cudaStream_t s,
                          const Composite *cmp = nullptr, const Input *staged_from = nullptr) {
    if (staged_from) {
        // I and alpha into their row-aligned copies (`in` describes the copies)
        const Input &o = *staged_from;
        StageList L;
        std::memset(&L, 0, sizeof L);
        L.local[0] = StageJob{o.I, const_cast<void *>(in.I), o.I_pitch * es, in.I_pitch * es,
                              3LL * o.w * es, o.h, 0};
        L.local[1] = StageJob{o.A, const_cast<void *>(in.A), o.A_pitch * es, in.A_pitch * es,
                              (long long)o.w * es, o.h, o.h};
        cudaError_t e = launch_stage_rows(dtype, L, 2, 2LL * o.h, s);
        if (e != cudaSuccess) return cuda_fail(e, "row-aligned copy of the inputs");
    }
    const int n = (int)lv.size();
    CoarseArgs ca;
    std::memset(&ca, 0, sizeof ca);
    ca.I = in.I;
    ca.I_pitch = in.I_pitch;
    ca.A = in.A;
    ca.A_pitch = in.A_pitch;
    ca.Iw = in.w;
    ca.Ih = in.h;
    ca.nlev = nc;
    for (int l = 0; l < nc; ++l) {
        ca.lw[l] = lv[l].w;
        ca.lh[l] = lv[l].h;
        ca.lk[l] = lv[l].k;
        ca.off[l] = ca.total;
        ca.total += lv[l].w * lv[l].h;
    }
    ca.eps = p.eps_r;
    ca.omega = p.omega;
    ca.init = p.init;
    ca.order = p.order;
    State src{};
    int buf = -1;
    if (nc == n) {
        ca.Fd = Fd;
        ca.Bd = Bd;
        ca.d_pitch = d_pitch;
        if (cmp) {
            ca.Bn = cmp->Bn;
            ca.In = cmp->In;
            ca.bn_pitch = cmp->bn_pitch;
            ca.in_pitch = cmp->in_pitch;
        }
    } else {
        src = state_in(ws.lev[0], lv[nc - 1].w, lv[nc - 1].h, es);
        buf = 0;
        ca.Fd = (void *)src.F;
        ca.Bd = (void *)src.B;
        ca.d_pitch = src.pitch;
    }
    cudaError_t e = launch_coarse(dtype, p.clamp, ca, s);
    if (e != cudaSuccess) return cuda_fail(e, "coarse kernel launch");

    int l = nc;
    // the run of small levels after the coarse ones, in one launch (Jacobi order)
    ConeArgs cone;
    const int m = cone_run(lv, nc, p);
    if (m >= nc && plan_cone(in, lv, nc, m, src, p, cone)) {
        State dst{};
        int nb = buf;
        if (m == n - 1) {
            cone.Fd = Fd;
            cone.Bd = Bd;
            cone.d_pitch = d_pitch;
            if (cmp) {
                cone.Bn = cmp->Bn;
                cone.In = cmp->In;
                cone.bn_pitch = cmp->bn_pitch;
                cone.in_pitch = cmp->in_pitch;
            }
        } else {
            nb = buf == 0 ? 1 : 0;
            dst = state_in(ws.lev[nb], lv[m].w, lv[m].h, es);
            cone.Fd = (void *)dst.F;
            cone.Bd = (void *)dst.B;
            cone.d_pitch = dst.pitch;
        }
        if ((e = launch_cone(dtype, p.clamp, cone, s)) != cudaSuccess) return cuda_fail(e, "small-level launch");
        src = dst;
        buf = nb;
        l = m + 1;
    }
    for (; l < n; ++l) {
        fg_status st = run_level(dtype, p, in, src, buf, lv[l].k, lv[l].w, lv[l].h, l == n - 1,
                                 Fd, Bd, d_pitch, ws, es, s, l == n - 1 ? cmp : nullptr);
        if (st != FG_OK) return st;
    }
    return FG_OK;
}

// Per-device stream on which launch sequences are captured into graphs.
cudaStream_t capture_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    const int d = current_device();
    if (d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[d] && cudaStreamCreateWithFlags(&streams[d], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[d] = nullptr;
    }
    return streams[d];
}

bool graphs_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("FGML_NO_GRAPH");
        return !(v && *v && *v != '0');
    }();
    return on;
}

fg_status estimate(const Input &in, int dtype, const fg_params &p, void *Fd, void *Bd,
                   long long d_pitch, cudaStream_t s, const Composite *cmp = nullptr) {
    const int es = dtype == kF32 ? 4 : 2;
    const std::vector<Level> lv = plan_levels(in.w, in.h, p);
    const int n = (int)lv.size();
    const int nc = coarse_levels(lv);   // levels run by the coarse kernel

    // workspace: every intermediate state, including extra passes of the top level
    size_t need = 0;
    if (nc < n) need = state_bytes(lv[nc - 1].w, lv[nc - 1].h, es);
    for (int l = nc; l < n; ++l) {
        const bool top = l == n - 1;
        if (!top || split_sweeps(lv[l].k).size() > 1)
            need = std::max(need, state_bytes(lv[l].w, lv[l].h, es));
    }
    Workspace &ws = workspace_for(s);
    // Rows off the 16-byte grid cannot be described by tensor maps: the level passes of a
    // large image then read a row-aligned copy of I and alpha (one copy kernel, 32 bytes
    // per pixel in FP32), or the input in place by per-lane copies (see needs_stage).
    const bool stage = n > nc && (long long)in.w * in.h > small_level_pixels() && needs_stage(in, es);
    const long long pI = ((3LL * in.w * es + 15) & ~15LL) / es, pA = (((long long)in.w * es + 15) & ~15LL) / es;
    const size_t offA = align256((size_t)(pI * es) * in.h);
    const size_t stage_need = stage ? offA + align256((size_t)(pA * es) * in.h) : 0;
    if ((need && (ws.lev[0].bytes < need || ws.lev[1].bytes < need)) || ws.align.bytes < stage_need) {
        // cached graphs point at the buffers about to be replaced
        cudaStreamSynchronize(s);
        clear_graphs(ws, s);
        fg_status st = ensure(ws.lev[0], need, s);
        if (st != FG_OK) return st;
        st = ensure(ws.lev[1], need, s);
        if (st != FG_OK) return st;
        st = ensure(ws.align, stage_need, s);
        if (st != FG_OK) return st;
    }
    Input run = in;
    if (stage) {
        run.I = ws.align.p;
        run.A = static_cast<char *>(ws.align.p) + offA;
        run.I_pitch = pI;
        run.A_pitch = pA;
        run.padded = true;
    }
    const Input *from = stage ? &in : nullptr;
    if (!graphs_enabled())
        return launch_sequence(run, dtype, p, lv, nc, Fd, Bd, d_pitch, ws, es, s, cmp, from);

    // the launch sequence depends on the pointers, pitches, sizes, dtype and parameters
    struct {
        const void *I, *A;
        void *F, *B;
        long long Ip, Ap, dp;
        int w, h, dtype;
        fg_params p;
        const void *Bn;
        void *In;
        long long bnp, inp;
    } sig;
    std::memset(&sig, 0, sizeof sig);
    sig.I = in.I;
    sig.A = in.A;
    sig.F = Fd;
    sig.B = Bd;
    sig.Ip = in.I_pitch;
    sig.Ap = in.A_pitch;
    sig.dp = d_pitch;
    sig.w = in.w;
    sig.h = in.h;
    sig.dtype = dtype;
    sig.p = p;
    if (cmp) {
        sig.Bn = cmp->Bn;
        sig.In = cmp->In;
        sig.bnp = cmp->bn_pitch;
        sig.inp = cmp->in_pitch;
    }
    const std::string key(reinterpret_cast<const char *>(&sig), sizeof sig);
    auto it = ws.graphs.find(key);
    if (it == ws.graphs.end()) {
        cudaStream_t cs = capture_stream();
        if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return launch_sequence(run, dtype, p, lv, nc, Fd, Bd, d_pitch, ws, es, s, cmp, from);
        }
        fg_status st = launch_sequence(run, dtype, p, lv, nc, Fd, Bd, d_pitch, ws, es, cs, cmp, from);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st != FG_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "capturing the launch sequence");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "instantiating the launch graph");
        evict_graphs(ws, s);
        it = ws.graphs.emplace(key, ex).first;
        ws.graph_order.push_back(key);
    }
    cudaError_t e = cudaGraphLaunch(it->second, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return FG_OK;
}

bool debug_checks() {
    const char *v = std::getenv("FGML_DEBUG");
    return v && *v && *v != '0';
}

// The input range check of FGML_DEBUG=1: counts the values of I and alpha outside [0, 1]
// or NaN into the device word *bad and returns FG_ERR_RANGE if there are any. It
// synchronises the stream.
fg_status range_check(const Input &in, int dtype, unsigned long long *bad, cudaStream_t s) {
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof h, s);
    if (e == cudaSuccess) e = launch_range_check(dtype, in.I, in.I_pitch, in.w, in.h, 3, bad, s);
    if (e == cudaSuccess) e = launch_range_check(dtype, in.A, in.A_pitch, in.w, in.h, 1, bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "input range check");
    if (h) return fail(FG_ERR_RANGE, "%llu values of I and alpha are outside [0, 1] or NaN", h);
    return FG_OK;
}

// FGML_DEBUG=1: every solve first checks that I and alpha hold values in [0, 1] (no NaN)
// and returns FG_ERR_RANGE otherwise; the counter lives in the stream's workspace.
fg_status check_inputs(const Input &in, int dtype, cudaStream_t s) {
    if (!debug_checks()) return FG_OK;
    Workspace &ws = workspace_for(s);
    fg_status st = ensure(ws.check, sizeof(unsigned long long), s);
    if (st != FG_OK) return st;
    return range_check(in, dtype, static_cast<unsigned long long *>(ws.check.p), s);
}

fg_params params_or_default(const fg_params *p) {
    fg_params d;
    fg_params_default(&d);
    return p ? *p : d;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

void fg_params_default(fg_params *p) {
    if (!p) return;
    p->eps_r = 5e-3f;
    p->omega = 0.1f;
    p->small_size = 32;
    p->small_iters = 10;
    p->big_iters = 2;
    p->order = FG_ORDER_JACOBI;
    p->clamp = 1;
    p->init = 0.f;
}

int fg_schedule(int w, int h, const fg_params *params, int *ws, int *hs, int *ks, int cap) {
    if (w < 1 || h < 1 || w > kMaxSide || h > kMaxSide) return -1;
    const fg_params p = params_or_default(params);
    const std::vector<Level> lv = plan_levels(w, h, p);
    if ((int)lv.size() > cap) return -1;
    for (size_t i = 0; i < lv.size(); ++i) {
        if (ws) ws[i] = lv[i].w;
        if (hs) hs[i] = lv[i].h;
        if (ks) ks[i] = lv[i].k;
    }
    return (int)lv.size();
}

fg_status fg_estimate(const fg_image *I, const fg_image *alpha, const fg_params *params,
                      fg_image *F, fg_image *B, void *stream) {
    g_err.clear();
    Range range("fg_estimate");
    fg_status st;
    if ((st = check_image(I, 3, "I")) != FG_OK) return st;
    if ((st = check_image(alpha, 1, "alpha")) != FG_OK) return st;
    if ((st = check_image(F, 3, "F")) != FG_OK) return st;
    if ((st = check_image(B, 3, "B")) != FG_OK) return st;
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    if (alpha->w != I->w || alpha->h != I->h || F->w != I->w || F->h != I->h ||
        B->w != I->w || B->h != I->h)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same size");
    if (alpha->dtype != I->dtype || F->dtype != I->dtype || B->dtype != I->dtype)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same dtype");
    if (F->row_pitch_bytes != B->row_pitch_bytes)
        return fail(FG_ERR_INVALID_ARG, "F and B must have the same row pitch");
    if (overlap(F, 3, B, 3) || overlap(F, 3, I, 3) || overlap(F, 3, alpha, 1) ||
        overlap(B, 3, I, 3) || overlap(B, 3, alpha, 1))
        return fail(FG_ERR_INVALID_ARG, "outputs overlap each other or the inputs");
    const int es = elem_size(I->dtype);
    Input in{I->ptr, alpha->ptr, I->row_pitch_bytes / es, alpha->row_pitch_bytes / es, I->w, I->h};
    if ((st = check_inputs(in, (int)I->dtype, (cudaStream_t)stream)) != FG_OK) return st;
    return estimate(in, (int)I->dtype, p, F->ptr, B->ptr, F->row_pitch_bytes / es,
                    (cudaStream_t)stream);
}

fg_status fg_estimate_composite(const fg_image *I, const fg_image *alpha, const fg_params *params,
                                fg_image *F, fg_image *B, const fg_image *B_new, fg_image *I_new,
                                void *stream) {
    g_err.clear();
    Range range("fg_estimate_composite");
    fg_status st;
    if ((st = check_image(B_new, 3, "B_new")) != FG_OK) return st;
    if ((st = check_image(I_new, 3, "I_new")) != FG_OK) return st;
    if ((st = check_image(I, 3, "I")) != FG_OK) return st;
    if ((st = check_image(alpha, 1, "alpha")) != FG_OK) return st;
    if ((st = check_image(F, 3, "F")) != FG_OK) return st;
    if ((st = check_image(B, 3, "B")) != FG_OK) return st;
    if (B_new->w != I->w || B_new->h != I->h || I_new->w != I->w || I_new->h != I->h)
        return fail(FG_ERR_INVALID_ARG, "B_new and I_new must have the size of I");
    if (B_new->dtype != I->dtype || I_new->dtype != I->dtype)
        return fail(FG_ERR_INVALID_ARG, "B_new and I_new must have the dtype of I");
    if (overlap(I_new, 3, I, 3) || overlap(I_new, 3, alpha, 1) || overlap(I_new, 3, F, 3) ||
        overlap(I_new, 3, B, 3) || overlap(I_new, 3, B_new, 3) || overlap(F, 3, B_new, 3) ||
        overlap(B, 3, B_new, 3))
        return fail(FG_ERR_INVALID_ARG, "I_new overlaps another image, or F or B overlaps B_new");
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    if (alpha->w != I->w || alpha->h != I->h || F->w != I->w || F->h != I->h ||
        B->w != I->w || B->h != I->h)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same size");
    if (alpha->dtype != I->dtype || F->dtype != I->dtype || B->dtype != I->dtype)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same dtype");
    if (F->row_pitch_bytes != B->row_pitch_bytes)
        return fail(FG_ERR_INVALID_ARG, "F and B must have the same row pitch");
    if (overlap(F, 3, B, 3) || overlap(F, 3, I, 3) || overlap(F, 3, alpha, 1) ||
        overlap(B, 3, I, 3) || overlap(B, 3, alpha, 1))
        return fail(FG_ERR_INVALID_ARG, "outputs overlap each other or the inputs");
    const int es = elem_size(I->dtype);
    Input in{I->ptr, alpha->ptr, I->row_pitch_bytes / es, alpha->row_pitch_bytes / es, I->w, I->h};
    if ((st = check_inputs(in, (int)I->dtype, (cudaStream_t)stream)) != FG_OK) return st;
    Composite c;
    c.Bn = B_new->ptr;
    c.In = I_new->ptr;
    c.bn_pitch = B_new->row_pitch_bytes / es;
    c.in_pitch = I_new->row_pitch_bytes / es;
    return estimate(in, (int)I->dtype, p, F->ptr, B->ptr, F->row_pitch_bytes / es,
                    (cudaStream_t)stream, &c);
}

}  // extern "C"

namespace {

// Host buffers in, host buffers out, on `s`: contiguous copies of I and alpha into the
// stream's staging buffers (a pitched copy from host memory runs at a fraction of the
// link's bandwidth when rows are a few KB), the solve (which first puts rows that are off
// the 16-byte grid onto it, on the device), contiguous copies of F and B back; `sync`
// waits for the stream.
fg_status estimate_host(const void *I, const void *alpha, int w, int h, fg_dtype dtype,
                        const fg_params *params, void *F, void *B, cudaStream_t s, bool sync) {
    g_err.clear();
    Range range("fg_estimate_host");
    if (!I || !alpha || !F || !B) return fail(FG_ERR_INVALID_ARG, "NULL host pointer");
    if (w < 1 || h < 1 || w > kMaxSide || h > kMaxSide)
        return fail(FG_ERR_INVALID_ARG, "size %dx%d outside [1, %d]", w, h, kMaxSide);
    if (dtype != FG_F32 && dtype != FG_BF16 && dtype != FG_F16)
        return fail(FG_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    const fg_params p = params_or_default(params);
    fg_status st = check_params(p);
    if (st != FG_OK) return st;
    const int es = elem_size(dtype);
    const size_t n = (size_t)w * h;
    const size_t bI = align256(3 * n * es), bA = align256(n * es), bO = bI;
    Workspace &ws = workspace_for(s);
    if ((st = ensure(ws.stage, bI + bA + 2 * bO, s)) != FG_OK) return st;
    char *dI = (char *)ws.stage.p, *dA = dI + bI, *dF = dA + bA, *dB = dF + bO;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dI, I, 3 * n * es, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy of I to the device");
    if ((e = cudaMemcpyAsync(dA, alpha, n * es, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy of alpha to the device");
    Input in{dI, dA, 3LL * w, (long long)w, w, h, false};
    if ((st = estimate(in, (int)dtype, p, dF, dB, 3LL * w, s)) != FG_OK) return st;
    if ((e = cudaMemcpyAsync(F, dF, 3 * n * es, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copy of F to the host");
    if ((e = cudaMemcpyAsync(B, dB, 3 * n * es, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copy of B to the host");
    if (sync && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return FG_OK;
}

}  // namespace

extern "C" {

fg_status fg_estimate_host(const void *I, const void *alpha, int w, int h, fg_dtype dtype,
                           const fg_params *params, void *F, void *B, void *stream) {
    return estimate_host(I, alpha, w, h, dtype, params, F, B, (cudaStream_t)stream, true);
}

fg_status fg_estimate_host_async(const void *I, const void *alpha, int w, int h, fg_dtype dtype,
                                 const fg_params *params, void *F, void *B, void *stream) {
    return estimate_host(I, alpha, w, h, dtype, params, F, B, (cudaStream_t)stream, false);
}

fg_status fg_level_pass(const fg_image *I, const fg_image *alpha, const fg_image *F_src,
                        const fg_image *B_src, int iters, const fg_params *params,
                        fg_image *F_dst, fg_image *B_dst, void *stream) {
    g_err.clear();
    fg_status st;
    if ((st = check_image(I, 3, "I")) != FG_OK) return st;
    if ((st = check_image(alpha, 1, "alpha")) != FG_OK) return st;
    if ((st = check_image(F_src, 3, "F_src")) != FG_OK) return st;
    if ((st = check_image(B_src, 3, "B_src")) != FG_OK) return st;
    if ((st = check_image(F_dst, 3, "F_dst")) != FG_OK) return st;
    if ((st = check_image(B_dst, 3, "B_dst")) != FG_OK) return st;
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    if (iters < 0) return fail(FG_ERR_INVALID_ARG, "iters must be >= 0");
    if (alpha->w != I->w || alpha->h != I->h)
        return fail(FG_ERR_INVALID_ARG, "I and alpha must have the same size");
    if (F_src->w != B_src->w || F_src->h != B_src->h || F_src->row_pitch_bytes != B_src->row_pitch_bytes)
        return fail(FG_ERR_INVALID_ARG, "F_src and B_src must have the same size and pitch");
    if (F_dst->w != B_dst->w || F_dst->h != B_dst->h || F_dst->row_pitch_bytes != B_dst->row_pitch_bytes)
        return fail(FG_ERR_INVALID_ARG, "F_dst and B_dst must have the same size and pitch");
    const fg_dtype dt = I->dtype;
    if (alpha->dtype != dt || F_src->dtype != dt || B_src->dtype != dt || F_dst->dtype != dt ||
        B_dst->dtype != dt)
        return fail(FG_ERR_INVALID_ARG, "all images must have the same dtype");
    if (overlap(F_dst, 3, B_dst, 3) || overlap(F_dst, 3, F_src, 3) || overlap(F_dst, 3, B_src, 3) ||
        overlap(B_dst, 3, F_src, 3) || overlap(B_dst, 3, B_src, 3) || overlap(F_dst, 3, I, 3) ||
        overlap(B_dst, 3, I, 3) || overlap(F_dst, 3, alpha, 1) || overlap(B_dst, 3, alpha, 1))
        return fail(FG_ERR_INVALID_ARG, "outputs overlap each other or the inputs");
    const int es = elem_size(dt);
    cudaStream_t s = (cudaStream_t)stream;
    Input in{I->ptr, alpha->ptr, I->row_pitch_bytes / es, alpha->row_pitch_bytes / es, I->w, I->h};
    // the sources' rows are readable up to their pitch, the last row included
    State src{F_src->ptr, B_src->ptr, F_src->row_pitch_bytes / es, F_src->w, F_src->h, true};
    const int w = F_dst->w, h = F_dst->h;
    Workspace &ws = workspace_for(s);
    if (split_sweeps(iters).size() > 1) {
        if ((st = ensure(ws.lev[0], state_bytes(w, h, es), s)) != FG_OK) return st;
        if ((st = ensure(ws.lev[1], state_bytes(w, h, es), s)) != FG_OK) return st;
    }
    int buf = -1;   // the source is caller memory
    return run_level((int)dt, p, in, src, buf, iters, w, h, true, F_dst->ptr, B_dst->ptr,
                     F_dst->row_pitch_bytes / es, ws, es, s);
}

fg_status fg_quality(const fg_image *F_est, const fg_image *F_gt, const fg_image *alpha_gt,
                     double *out, void *stream) {
    g_err.clear();
    Range range("fg_quality");
    fg_status st;
    if ((st = check_image(F_est, 3, "F_est")) != FG_OK) return st;
    if ((st = check_image(F_gt, 3, "F_gt")) != FG_OK) return st;
    if ((st = check_image(alpha_gt, 1, "alpha_gt")) != FG_OK) return st;
    if (!out) return fail(FG_ERR_INVALID_ARG, "out is NULL");
    if (F_gt->w != F_est->w || F_gt->h != F_est->h || alpha_gt->w != F_est->w || alpha_gt->h != F_est->h)
        return fail(FG_ERR_INVALID_ARG, "F_est, F_gt and alpha_gt must have the same size");
    const fg_dtype dt = F_est->dtype;
    if (F_gt->dtype != dt || alpha_gt->dtype != dt)
        return fail(FG_ERR_INVALID_ARG, "F_est, F_gt and alpha_gt must have the same dtype");
    const int es = elem_size(dt);
    cudaStream_t s = (cudaStream_t)stream;
    Workspace &ws = workspace_for(s);
    const long long nb = quality_blocks(F_est->w, F_est->h);
    if ((st = ensure(ws.aux, (size_t)(3 * nb + 3) * sizeof(double), s)) != FG_OK) return st;
    QualityArgs q;
    std::memset(&q, 0, sizeof q);
    q.Fe = F_est->ptr;
    q.Fg = F_gt->ptr;
    q.A = alpha_gt->ptr;
    q.fe_pitch = F_est->row_pitch_bytes / es;
    q.fg_pitch = F_gt->row_pitch_bytes / es;
    q.a_pitch = alpha_gt->row_pitch_bytes / es;
    q.w = F_est->w;
    q.h = F_est->h;
    // sampled Gaussian (normalised to sum 1) and its derivative, sigma = 1.4 (Section IV-C)
    const double sigma = 1.4;
    double g[2 * kQualityRadius + 1], sum = 0.0;
    for (int k = -kQualityRadius; k <= kQualityRadius; ++k)
        sum += g[k + kQualityRadius] = std::exp(-0.5 * k * k / (sigma * sigma));
    for (int k = -kQualityRadius; k <= kQualityRadius; ++k) {
        const double gk = g[k + kQualityRadius] / sum;
        q.g[k + kQualityRadius] = (float)gk;
        q.dg[k + kQualityRadius] = (float)(-k / (sigma * sigma) * gk);
    }
    q.partials = static_cast<double *>(ws.aux.p);
    double *dout = q.partials + 3 * nb;
    cudaError_t e = launch_quality((int)dt, q, dout, s);
    if (e != cudaSuccess) return cuda_fail(e, "quality kernel launch");
    e = cudaMemcpyAsync(out, dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "quality result copy");
    return FG_OK;
}

fg_status fg_minimiser_cg(const fg_image *I, const fg_image *alpha, const fg_params *params,
                          double *F, double *B, int max_iters, double rel_tol, int *iters,
                          double *rel_residual, void *stream) {
    g_err.clear();
    Range range("fg_minimiser_cg");
    fg_status st;
    if ((st = check_image(I, 3, "I")) != FG_OK) return st;
    if ((st = check_image(alpha, 1, "alpha")) != FG_OK) return st;
    if (alpha->w != I->w || alpha->h != I->h || alpha->dtype != I->dtype)
        return fail(FG_ERR_INVALID_ARG, "I and alpha must have the same size and dtype");
    if (!F || !B) return fail(FG_ERR_INVALID_ARG, "F or B is NULL");
    if (max_iters < 0 || !(rel_tol >= 0.0))
        return fail(FG_ERR_INVALID_ARG, "max_iters must be >= 0 and rel_tol >= 0");
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    const int es = elem_size(I->dtype), w = I->w, h = I->h;
    const long long n = (long long)w * h;
    const size_t vec = (size_t)(6 * n) * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    Workspace &ws = workspace_for(s);
    const int nb = cg_blocks(w, h);
    const size_t vec_al = align256(vec);
    const size_t need = 6 * vec_al + align256((size_t)3 * nb * sizeof(double)) + sizeof(CgScalars);
    if ((st = ensure(ws.cg, need, s)) != FG_OK) return st;
    char *base = static_cast<char *>(ws.cg.p);
    CgArgs a;
    std::memset(&a, 0, sizeof a);
    a.I = I->ptr;
    a.A = alpha->ptr;
    a.I_pitch = I->row_pitch_bytes / es;
    a.A_pitch = alpha->row_pitch_bytes / es;
    a.w = w;
    a.h = h;
    a.eps = p.eps_r;
    a.omega = p.omega;
    a.x = reinterpret_cast<double *>(base);
    a.r = reinterpret_cast<double *>(base + vec_al);
    a.z = reinterpret_cast<double *>(base + 2 * vec_al);
    a.q = reinterpret_cast<double *>(base + 3 * vec_al);
    double *pv[2] = {reinterpret_cast<double *>(base + 4 * vec_al),
                     reinterpret_cast<double *>(base + 5 * vec_al)};
    a.partials = reinterpret_cast<double *>(base + 6 * vec_al);
    a.sc = reinterpret_cast<CgScalars *>(base + 6 * vec_al + align256((size_t)3 * nb * sizeof(double)));
    const size_t half = vec / 2;
    cudaError_t e = cudaMemcpyAsync(a.x, F, half, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.x + 3 * n, B, half, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cg_start((int)I->dtype, a, pv[0], s);
    CgScalars hs;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, a.sc, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "conjugate gradients start");
    int it = 0, cur = 0;
    const double stop = rel_tol * rel_tol * hs.bb;
    while (it < max_iters && hs.rr > stop) {
        const int chunk = std::min(32, max_iters - it);
        for (int k = 0; k < chunk && e == cudaSuccess; ++k) {
            e = cg_iterate((int)I->dtype, a, pv[cur], pv[cur ^ 1], s);
            cur ^= 1;
        }
        it += chunk;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, a.sc, sizeof hs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "conjugate gradients iteration");
        if (!std::isfinite(hs.rr)) return fail(FG_ERR_RANGE, "conjugate gradients diverged (is alpha constant?)");
    }
    // the reported residual is recomputed from x, not the recursively updated one
    e = cg_true_residual((int)I->dtype, a, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, a.x, half, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B, a.x + 3 * n, half, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, a.sc, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "conjugate gradients result");
    if (iters) *iters = it;
    if (rel_residual) *rel_residual = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : std::sqrt(hs.rr);
    return FG_OK;
}

fg_status fg_sync(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int code = 0;
    e = read_and_clear_device_error(&code, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (code) return fail(FG_ERR_TIMEOUT, "a bounded device-side wait gave up (code %d)", code);
    return FG_OK;
}

fg_status fg_release_workspace(void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    Workspace w;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws.find({current_device(), s});
        if (it == g_ws.end()) return FG_OK;
        w = it->second;
        g_ws.erase(it);
    }
    cudaStreamSynchronize(s);
    clear_graphs(w, s);
    cudaFree(w.lev[0].p);
    cudaFree(w.lev[1].p);
    cudaFree(w.stage.p);
    cudaFree(w.batch.p);
    cudaFree(w.worklist.p);
    cudaFree(w.aux.p);
    cudaFree(w.cg.p);
    cudaFree(w.check.p);
    cudaFree(w.align.p);
    return FG_OK;
}

const char *fg_last_error(void) { return g_err.c_str(); }

const char *fg_version(void) { return "fgml 0.1 (sm_103a)"; }

}  // extern "C"

// ====================================================== no-allocation variant
//
// fg_estimate_noalloc runs the same launch sequence as fg_estimate, but its intermediate
// pyramid levels live in a fixed array compiled into the library instead of a workspace
// taken with cudaMalloc. It serves callers that must not allocate device memory from
// inside this library: processes whose device memory is fully reserved up front by their
// own pool or budget, and hot loops that cannot afford cudaMalloc's implicit device-wide
// synchronisation. The array exists once per device that loads the library and stays
// allocated until the process exits.

namespace {

// Two level buffers of 32 MiB each (room for every intermediate level of an FP32 image of
// up to about 5.6 megapixels with the default schedule, twice that in BF16/FP16), then
// 256 bytes for the counter of the FGML_DEBUG=1 input range check.
constexpr size_t kNoAllocLevelBytes = 32ull << 20;
constexpr size_t kNoAllocScratchBytes = 2 * kNoAllocLevelBytes + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The device address of the array, looked up once per device and context: the host-side
// symbol is only a stand-in. A context is identified by the driver's process-unique
// context id, so after cudaDeviceReset (a new primary context, the module loaded again)
// the address is looked up again rather than reused.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct NoallocAddr {
    unsigned long long ctx_id = 0;   // 0: not looked up (or no id available)
    void *p = nullptr;
};
std::mutex g_noalloc_mu;
NoallocAddr g_noalloc_addr[64];

// Unique id of the calling thread's current context, or 0 if there is none or the driver
// does not report ids (then every call looks the address up).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

fg_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(FG_ERR_UNSUPPORTED, "device index %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocAddr &c = g_noalloc_addr[dev];
    const unsigned long long id = current_ctx_id();
    if (!c.p || !id || c.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
        c.p = p;
        c.ctx_id = current_ctx_id();   // the lookup may have made the primary context current
    }
    *out = c.p;
    return FG_OK;
}

}  // namespace

extern "C" fg_status fg_estimate_noalloc(const fg_image *I, const fg_image *alpha,
                                         const fg_params *params, fg_image *F, fg_image *B,
                                         void *stream) {
    g_err.clear();
    Range range("fg_estimate_noalloc");
    fg_status st;
    if ((st = check_image(I, 3, "I")) != FG_OK) return st;
    if ((st = check_image(alpha, 1, "alpha")) != FG_OK) return st;
    if ((st = check_image(F, 3, "F")) != FG_OK) return st;
    if ((st = check_image(B, 3, "B")) != FG_OK) return st;
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    if (alpha->w != I->w || alpha->h != I->h || F->w != I->w || F->h != I->h ||
        B->w != I->w || B->h != I->h)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same size");
    if (alpha->dtype != I->dtype || F->dtype != I->dtype || B->dtype != I->dtype)
        return fail(FG_ERR_INVALID_ARG, "I, alpha, F and B must have the same dtype");
    if (F->row_pitch_bytes != B->row_pitch_bytes)
        return fail(FG_ERR_INVALID_ARG, "F and B must have the same row pitch");
    if (overlap(F, 3, B, 3) || overlap(F, 3, I, 3) || overlap(F, 3, alpha, 1) ||
        overlap(B, 3, I, 3) || overlap(B, 3, alpha, 1))
        return fail(FG_ERR_INVALID_ARG, "outputs overlap each other or the inputs");

    const int dtype = (int)I->dtype;
    const int es = elem_size(I->dtype);
    const Input in{I->ptr, alpha->ptr, I->row_pitch_bytes / es, alpha->row_pitch_bytes / es,
                   I->w, I->h};
    const std::vector<Level> lv = plan_levels(in.w, in.h, p);
    const int n = (int)lv.size();
    const int nc = coarse_levels(lv);
    size_t need = 0;   // bytes of one level buffer
    if (nc < n) need = state_bytes(lv[nc - 1].w, lv[nc - 1].h, es);
    for (int l = nc; l < n; ++l)
        if (l != n - 1 || split_sweeps(lv[l].k).size() > 1)
            need = std::max(need, state_bytes(lv[l].w, lv[l].h, es));
    if (need > kNoAllocLevelBytes)
        return fail(FG_ERR_INVALID_ARG,
                    "%dx%d needs two %zu-byte level buffers; the no-allocation scratch holds "
                    "two of %zu bytes (use fg_estimate)",
                    in.w, in.h, need, kNoAllocLevelBytes);

    void *scratch = nullptr;
    if ((st = noalloc_scratch(&scratch)) != FG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (debug_checks()) {
        // the counter is the scratch's tail; range_check clears it before counting
        auto *bad = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) +
                                                           2 * kNoAllocLevelBytes);
        if ((st = range_check(in, dtype, bad, s)) != FG_OK) return st;
    }
    // Every byte a kernel reads from the level buffers was written earlier in this call,
    // so nothing needs clearing between calls. Inputs whose rows are off the 16-byte grid
    // are read in place (no row-aligned copy, which would need more memory).
    Workspace ws;
    ws.lev[0].p = scratch;
    ws.lev[0].bytes = kNoAllocLevelBytes;
    ws.lev[1].p = static_cast<char *>(scratch) + kNoAllocLevelBytes;
    ws.lev[1].bytes = kNoAllocLevelBytes;
    return launch_sequence(in, dtype, p, lv, nc, F->ptr, B->ptr, F->row_pitch_bytes / es, ws, es,
                           s);
}

// ====================================================== work-list batches

namespace {

constexpr int kBatchRegionCap = 48 * 1024;     // per-warp shared memory of the batch kernel at most
constexpr int kBatchChunkCap = 13 * 1024;      // chunk slot size that keeps two blocks per SM
constexpr long long kBatchWaitNs = 2000000000; // bound of one dependency wait (2 s)

// Rows per strip of a batch pass: a few waves of the persistent grid per level.
// Strip shape of the work-list passes: about `per_sm` strips per SM for a level, within
// [lo, hi] rows. The default comes from FGML_BATCH_STRIPS="per_sm,lo,hi" or the built-in
// {4, 8, 64}; fg_autotune_batch replaces it with the fastest measured candidate.
struct BatchStrips {
    int per_sm, lo, hi;
};
constexpr BatchStrips kStripCandidates[] = {{4, 28, 124}, {2, 60, 252}, {8, 28, 124}, {3, 44, 188},
                                            {6, 28, 92}, {2, 28, 124}};
std::mutex g_strips_mu;
BatchStrips g_strips = [] {
    BatchStrips v = kStripCandidates[0];
    const char *e = std::getenv("FGML_BATCH_STRIPS");
    int a, b, c;
    if (e && std::sscanf(e, "%d,%d,%d", &a, &b, &c) == 3 && a > 0 && b > 0 && c >= b) v = {a, b, c};
    return v;
}();

// FGML_TUNE_CACHE=path keeps the autotuned strip shape per GPU model across processes:
// one line per model, "<device name>\t<per_sm>,<lo>,<hi>".
std::string device_name() {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, current_device()) != cudaSuccess) return "unknown";
    return prop.name;
}

bool g_strips_cache_read = false;

void read_tune_cache() {   // with g_strips_mu held
    g_strips_cache_read = true;
    const char *path = std::getenv("FGML_TUNE_CACHE");
    if (!path || !*path || std::getenv("FGML_BATCH_STRIPS")) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    const std::string want = device_name();
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char *tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        int a, b, c;
        if (want == line && std::sscanf(tab + 1, "%d,%d,%d", &a, &b, &c) == 3 && a > 0 && b > 0 && c >= b)
            g_strips = {a, b, c};
    }
    std::fclose(f);
}

void write_tune_cache(const BatchStrips &v) {
    const char *path = std::getenv("FGML_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string me = device_name();
    std::vector<std::string> keep;
    if (FILE *f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof line, f)) {
            const char *tab = std::strchr(line, '\t');
            if (tab && std::string(line, (size_t)(tab - line)) == me) continue;
            keep.push_back(line);
        }
        std::fclose(f);
    }
    if (FILE *f = std::fopen(path, "w")) {
        for (const std::string &l : keep) std::fputs(l.c_str(), f);
        std::fprintf(f, "%s\t%d,%d,%d\n", me.c_str(), v.per_sm, v.lo, v.hi);
        std::fclose(f);
    }
}

int batch_strip_rows(int w, int h, const BatchStrips *force = nullptr) {
    BatchStrips v;
    if (force) {
        v = *force;
    } else {
        std::lock_guard<std::mutex> lk(g_strips_mu);
        if (!g_strips_cache_read) read_tune_cache();
        v = g_strips;
    }
    const int nx = (w + level_pass_strip_width() - 1) / level_pass_strip_width();
    const long long target = (long long)sm_count() * v.per_sm;
    long long r = ((long long)h * nx + target - 1) / target;
    r = std::min<long long>(std::max<long long>(r, v.lo), v.hi);
    return (int)((r + 3) / 4 * 4);   // whole four-row chunks with the two halo rows each side
}

PassArgs batch_pass_args(const fg_params &p, const Input &in, const State &src, void *Fd,
                         void *Bd, long long d_pitch, int w, int h,
                         const BatchStrips *strips = nullptr) {
    PassArgs a;
    std::memset(&a, 0, sizeof a);
    a.I = in.I;
    a.I_pitch = in.I_pitch;
    a.A = in.A;
    a.A_pitch = in.A_pitch;
    a.Iw = in.w;
    a.Ih = in.h;
    a.Fs = src.F;
    a.Bs = src.B;
    a.s_pitch = src.pitch;
    a.sw = src.w;
    a.sh = src.h;
    a.Fd = Fd;
    a.Bd = Bd;
    a.d_pitch = d_pitch;
    a.w = w;
    a.h = h;
    a.eps = p.eps_r;
    a.omega = p.omega;
    a.strip_h = batch_strip_rows(w, h, strips);
    a.n_xstrips = (w + level_pass_strip_width() - 1) / level_pass_strip_width();
    a.n_warps = a.n_xstrips * ((h + a.strip_h - 1) / a.strip_h);
    return a;
}

fg_status batch_launch(int dtype, int clamp, BatchLaunch &b, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = launch_tile_batch(dtype, clamp, b, s, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel occupancy");
    if (per_sm < 1) return fail(FG_ERR_CUDA, "batch kernel does not fit on an SM");
    b.blocks = std::max(1, std::min(per_sm * sm_count(),
                                     (b.n_items + level_pass_warps_per_block() - 1) /
                                         level_pass_warps_per_block()));
    e = launch_tile_batch(dtype, clamp, b, s, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    return FG_OK;
}

// Bytes of each of the two buffers that hold an image's intermediate levels (0: none).
size_t image_level_bytes(const std::vector<Level> &lv, int nc, int es) {
    const int nl = (int)lv.size();
    size_t need = 0;
    if (nc < nl) need = state_bytes(lv[nc - 1].w, lv[nc - 1].h, es);
    for (int l = nc; l < nl; ++l)
        if (l != nl - 1 || split_sweeps(lv[l].k).size() > 1)
            need = std::max(need, state_bytes(lv[l].w, lv[l].h, es));
    return align256(need);
}

// One image's share of a work list: its coarse levels, then its level passes in order,
// over intermediate-level buffers and outputs fixed when it is planned. Pass j reads what
// pass j - 1 wrote (Algorithm 1: each level starts from the one below).
struct ImagePlan {
    CoarseArgs coarse;
    std::vector<BatchDesc> passes;
};

// Plans image `in` (levels lv, the first nc in the coarse kernel) writing the finest
// level to (Fd, Bd, d_pitch), with the intermediate levels ping-ponged in lev0 / lev1
// (`need` bytes each). False when a 16-bit pass would need per-lane copies off the 4-byte
// grid (no chunk layout); rows on the 16-byte grid always plan.
bool plan_image(int dtype, const fg_params &p, const Input &in, const std::vector<Level> &lv, int nc,
                void *Fd, void *Bd, long long d_pitch, void *lev0, void *lev1, size_t need,
                ImagePlan &out, const BatchStrips *strips = nullptr) {
    const int es = dtype == kF32 ? 4 : 2, nl = (int)lv.size();
    Buf b0{lev0, need}, b1{lev1, need};
    const Buf *bufs[2] = {&b0, &b1};
    CoarseArgs &ca = out.coarse;
    std::memset(&ca, 0, sizeof ca);
    ca.I = in.I;
    ca.I_pitch = in.I_pitch;
    ca.A = in.A;
    ca.A_pitch = in.A_pitch;
    ca.Iw = in.w;
    ca.Ih = in.h;
    ca.nlev = nc;
    for (int l = 0; l < nc; ++l) {
        ca.lw[l] = lv[l].w;
        ca.lh[l] = lv[l].h;
        ca.lk[l] = lv[l].k;
        ca.off[l] = ca.total;
        ca.total += lv[l].w * lv[l].h;
    }
    ca.eps = p.eps_r;
    ca.omega = p.omega;
    ca.init = p.init;
    State src{};
    int buf = -1;
    if (nc == nl) {
        ca.Fd = Fd;
        ca.Bd = Bd;
        ca.d_pitch = d_pitch;
    } else {
        src = state_in(b0, lv[nc - 1].w, lv[nc - 1].h, es);
        buf = 0;
        ca.Fd = (void *)src.F;
        ca.Bd = (void *)src.B;
        ca.d_pitch = src.pitch;
    }
    out.passes.clear();
    for (int l = nc; l < nl; ++l) {
        const std::vector<int> sweeps = split_sweeps(lv[l].k);
        for (size_t j = 0; j < sweeps.size(); ++j) {
            const bool to_caller = l == nl - 1 && j + 1 == sweeps.size();
            const int w = lv[l].w, h = lv[l].h;
            void *F = Fd, *B = Bd;
            long long dp = d_pitch;
            State dst{};
            int nb = buf;
            if (!to_caller) {
                nb = buf == 0 ? 1 : 0;
                dst = state_in(*bufs[nb], w, h, es);
                F = (void *)dst.F;
                B = (void *)dst.B;
                dp = dst.pitch;
            }
            BatchDesc d;
            std::memset(&d, 0, sizeof d);
            d.a = batch_pass_args(p, in, src, F, B, dp, w, h, strips);
            d.iters = sweeps[j];
            d.dep = out.passes.empty() ? -1 : (int)out.passes.size() - 1;
            d.dep_count = out.passes.empty() ? 0 : out.passes.back().a.n_warps;
            if (!plan_chunks(dtype, in, src, d.a, d.maps, kBatchChunkCap)) return false;
            out.passes.push_back(d);
            if (!to_caller) {
                src = dst;
                buf = nb;
            }
        }
    }
    return true;
}

// A work list: the coarse launch's images, then the pass descriptors and their strips.
struct WorkList {
    std::vector<CoarseArgs> coarse;
    std::vector<BatchDesc> descs;
    std::vector<std::vector<int>> parts;   // descriptor indices of each part, in order
    std::vector<BatchItem> items;
    int max_total = 0, region = 0;
};

// Adds passes [first, last) of `plan`, and its coarse levels when with_coarse (run by the
// coarse launch before the work list). Pass `first` waits for nothing: the passes before
// it are done, in earlier launches or in this one's coarse launch.
void worklist_add(WorkList &L, const ImagePlan &plan, bool with_coarse, int first, int last) {
    if (with_coarse) {
        L.coarse.push_back(plan.coarse);
        L.max_total = std::max(L.max_total, plan.coarse.total);
    }
    std::vector<int> ix;
    for (int j = first; j < last; ++j) {
        BatchDesc d = plan.passes[j];
        d.dep = ix.empty() ? -1 : ix.back();
        d.dep_count = ix.empty() ? 0 : L.descs[ix.back()].a.n_warps;
        ix.push_back((int)L.descs.size());
        L.descs.push_back(d);
    }
    if (!ix.empty()) L.parts.push_back(std::move(ix));
}

// Every warp's region holds two chunks of the largest pass; smaller passes keep as many
// chunks in flight as fit (at most three). Items are interleaved by rank (every part's
// first pass, then every part's second ...), so that the strips a strip waits for were
// all handed out before it.
fg_status worklist_finish(WorkList &L) {
    int chunk_max = 0;
    for (const BatchDesc &d : L.descs) chunk_max = std::max(chunk_max, d.a.tile_chunk);
    L.region = (2 * chunk_max + 127) & ~127;   // 128-byte aligned, as tensor copies into it require
    if (L.region > kBatchRegionCap) return fail(FG_ERR_CUDA, "batch region %d exceeds the cap", L.region);
    long long nitems = 0;
    for (BatchDesc &d : L.descs) {
        d.a.tile_slots = std::min(kBatchMaxSlots, L.region / std::max(1, d.a.tile_chunk));
        nitems += d.a.n_warps;
    }
    if (nitems > (1LL << 30)) return fail(FG_ERR_INVALID_ARG, "batch too large");
    L.items.clear();
    L.items.reserve((size_t)nitems);
    for (size_t rank = 0;; ++rank) {
        bool any = false;
        for (const std::vector<int> &part : L.parts) {
            if (rank >= part.size()) continue;
            any = true;
            const int dix = part[rank];
            for (int wi = 0; wi < L.descs[dix].a.n_warps; ++wi) L.items.push_back(BatchItem{dix, wi});
        }
        if (!any) break;
    }
    return FG_OK;
}

// Device copy of a work list: [row-aligned copy jobs][coarse args][descs][items][counters].
struct WorkListLayout {
    size_t off_jobs, off_coarse, off_desc, off_items, off_cnt, bytes;
};

WorkListLayout worklist_layout(const WorkList &L, size_t njobs) {
    WorkListLayout o;
    o.off_jobs = 0;
    o.off_coarse = align256(njobs * sizeof(StageJob));
    o.off_desc = align256(o.off_coarse + L.coarse.size() * sizeof(CoarseArgs));
    o.off_items = align256(o.off_desc + L.descs.size() * sizeof(BatchDesc));
    o.off_cnt = align256(o.off_items + L.items.size() * sizeof(BatchItem));
    o.bytes = align256(o.off_cnt + (1 + L.descs.size()) * sizeof(int));
    return o;
}

std::vector<char> worklist_blob(const WorkList &L, const std::vector<StageJob> &jobs,
                                const WorkListLayout &o) {
    std::vector<char> blob(o.bytes, 0);
    if (!jobs.empty()) std::memcpy(blob.data() + o.off_jobs, jobs.data(), jobs.size() * sizeof(StageJob));
    if (!L.coarse.empty())
        std::memcpy(blob.data() + o.off_coarse, L.coarse.data(), L.coarse.size() * sizeof(CoarseArgs));
    if (!L.descs.empty())
        std::memcpy(blob.data() + o.off_desc, L.descs.data(), L.descs.size() * sizeof(BatchDesc));
    if (!L.items.empty())
        std::memcpy(blob.data() + o.off_items, L.items.data(), L.items.size() * sizeof(BatchItem));
    return blob;
}

// The launches of one work list whose device copy is at `wl`: counters cleared, the
// row-aligned copies, the coarse levels of its images, the strips.
fg_status worklist_enqueue(int dtype, int clamp, const WorkList &L, const WorkListLayout &o,
                           size_t njobs, long long stage_rows, char *wl, cudaStream_t q) {
    cudaError_t e = cudaMemsetAsync(wl + o.off_cnt, 0, (1 + L.descs.size()) * sizeof(int), q);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the work-list counters");
    if (njobs) {
        StageList S;
        std::memset(&S, 0, sizeof S);
        S.dev = reinterpret_cast<const StageJob *>(wl + o.off_jobs);
        e = launch_stage_rows(dtype, S, (int)njobs, stage_rows, q);
        if (e != cudaSuccess) return cuda_fail(e, "row-aligned copies of the batch inputs");
    }
    if (!L.coarse.empty()) {
        e = launch_coarse_batch(dtype, clamp, reinterpret_cast<const CoarseArgs *>(wl + o.off_coarse),
                                (int)L.coarse.size(), L.max_total, q);
        if (e != cudaSuccess) return cuda_fail(e, "batched coarse kernel launch");
    }
    if (L.items.empty()) return FG_OK;
    BatchLaunch b;
    b.descs = reinterpret_cast<const BatchDesc *>(wl + o.off_desc);
    b.items = reinterpret_cast<const BatchItem *>(wl + o.off_items);
    b.n_items = (int)L.items.size();
    b.counters = reinterpret_cast<int *>(wl + o.off_cnt);
    b.wait_ns = kBatchWaitNs;
    b.slot_bytes = 0;
    b.region = L.region;
    return batch_launch(dtype, clamp, b, q);
}

}  // namespace

extern "C" fg_status fg_estimate_batch(int n, const fg_image *I, const fg_image *alpha,
                                       const fg_params *params, fg_image *F, fg_image *B,
                                       void *stream) {
    g_err.clear();
    Range range("fg_estimate_batch");
    if (n < 1 || !I || !alpha || !F || !B) return fail(FG_ERR_INVALID_ARG, "empty batch or NULL array");
    fg_status st;
    const fg_params p = params_or_default(params);
    if ((st = check_params(p)) != FG_OK) return st;
    const fg_dtype dt = I[0].dtype;
    for (int i = 0; i < n; ++i) {
        char nm[32];
        snprintf(nm, sizeof nm, "I[%d]", i);
        if ((st = check_image(&I[i], 3, nm)) != FG_OK) return st;
        snprintf(nm, sizeof nm, "alpha[%d]", i);
        if ((st = check_image(&alpha[i], 1, nm)) != FG_OK) return st;
        snprintf(nm, sizeof nm, "F[%d]", i);
        if ((st = check_image(&F[i], 3, nm)) != FG_OK) return st;
        snprintf(nm, sizeof nm, "B[%d]", i);
        if ((st = check_image(&B[i], 3, nm)) != FG_OK) return st;
        if (alpha[i].w != I[i].w || alpha[i].h != I[i].h || F[i].w != I[i].w || F[i].h != I[i].h ||
            B[i].w != I[i].w || B[i].h != I[i].h)
            return fail(FG_ERR_INVALID_ARG, "image %d: I, alpha, F and B differ in size", i);
        if (I[i].dtype != dt || alpha[i].dtype != dt || F[i].dtype != dt || B[i].dtype != dt)
            return fail(FG_ERR_INVALID_ARG, "image %d: every image of a batch has one dtype", i);
        if (F[i].row_pitch_bytes != B[i].row_pitch_bytes)
            return fail(FG_ERR_INVALID_ARG, "image %d: F and B must have the same row pitch", i);
        if (overlap(&F[i], 3, &B[i], 3) || overlap(&F[i], 3, &I[i], 3) ||
            overlap(&F[i], 3, &alpha[i], 1) || overlap(&B[i], 3, &I[i], 3) ||
            overlap(&B[i], 3, &alpha[i], 1))
            return fail(FG_ERR_INVALID_ARG, "image %d: outputs overlap each other or the inputs", i);
    }
    const int dtype = (int)dt, es = elem_size(dt);
    cudaStream_t s = (cudaStream_t)stream;

    struct Img {
        Input in;
        Input orig;            // the caller's input (in: its row-aligned copy when staged)
        std::vector<Level> lv;
        int nc;
        size_t need;
        size_t buf_off;
        bool stage;            // rows off the 16-byte grid: levels read a row-aligned copy
        size_t stage_off, stage_offA;
        long long pI, pA;      // pitches of the copy (elements)
    };
    std::vector<Img> im(n);
    bool zero_sweeps = false;
    size_t buf_total = 0;
    for (int i = 0; i < n; ++i) {
        Img &m = im[i];
        m.in = Input{I[i].ptr, alpha[i].ptr, I[i].row_pitch_bytes / es, alpha[i].row_pitch_bytes / es,
                     I[i].w, I[i].h};
        m.orig = m.in;
        m.lv = plan_levels(m.in.w, m.in.h, p);
        m.nc = coarse_levels(m.lv);
        const int nl = (int)m.lv.size();
        for (int l = m.nc; l < nl; ++l)
            if (m.lv[l].k == 0) zero_sweeps = true;
        m.need = image_level_bytes(m.lv, m.nc, es);
        m.buf_off = buf_total;
        buf_total += 2 * m.need;
        m.stage = m.nc < nl && needs_stage(m.in, es);
        if (m.stage) {
            m.pI = ((3LL * m.in.w * es + 15) & ~15LL) / es;
            m.pA = (((long long)m.in.w * es + 15) & ~15LL) / es;
            m.stage_off = buf_total;
            m.stage_offA = align256((size_t)(m.pI * es) * m.in.h);
            buf_total += m.stage_offA + align256((size_t)(m.pA * es) * m.in.h);
        }
    }
    if (zero_sweeps || p.order != FG_ORDER_JACOBI) {
        // levels without sweeps are plain resizes, and the work-list kernel runs the Jacobi
        // order only; run such parameter sets image by image
        for (int i = 0; i < n; ++i)
            if ((st = estimate(im[i].in, dtype, p, F[i].ptr, B[i].ptr, F[i].row_pitch_bytes / es, s)) != FG_OK)
                return st;
        return FG_OK;
    }

    // A repeated batch (same images, outputs, sizes, dtype, parameters and strip shape)
    // replays the launch graph captured for it: no descriptors are built or uploaded again.
    Workspace &wsb = workspace_for(s);
    std::string key;
    if (graphs_enabled()) {
        BatchStrips strips;
        {
            std::lock_guard<std::mutex> lk(g_strips_mu);
            if (!g_strips_cache_read) read_tune_cache();
            strips = g_strips;
        }
        key.assign("batch", 5);
        auto put = [&](const void *v, size_t k) { key.append(static_cast<const char *>(v), k); };
        put(&n, sizeof n);
        put(&p, sizeof p);
        put(&strips, sizeof strips);
        for (int i = 0; i < n; ++i) {
            const fg_image *four[4] = {&I[i], &alpha[i], &F[i], &B[i]};
            for (const fg_image *x : four) {   // fields only, no padding
                put(&x->ptr, sizeof x->ptr);
                put(&x->w, sizeof x->w);
                put(&x->h, sizeof x->h);
                put(&x->row_pitch_bytes, sizeof x->row_pitch_bytes);
                put(&x->dtype, sizeof x->dtype);
            }
            const char stg = im[i].stage ? 1 : 0;
            put(&stg, 1);
        }
        auto it = wsb.graphs.find(key);
        if (it != wsb.graphs.end()) {
            cudaError_t e = cudaGraphLaunch(it->second, s);
            if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
            return FG_OK;
        }
        auto seen = std::find(wsb.batch_seen.begin(), wsb.batch_seen.end(), key);
        if (seen == wsb.batch_seen.end()) {   // first sight: launch directly, remember it
            if (wsb.batch_seen.size() >= kMaxGraphs) wsb.batch_seen.erase(wsb.batch_seen.begin());
            wsb.batch_seen.push_back(key);
            key.clear();
        } else {
            wsb.batch_seen.erase(seen);
        }
    }

    Workspace &ws = wsb;
    if (ws.batch.bytes < buf_total + 256) {
        // cached graphs may point into the buffer about to be replaced
        cudaStreamSynchronize(s);
        clear_graphs(ws, s);
    }
    if ((st = ensure(ws.batch, buf_total + 256, s)) != FG_OK) return st;
    char *bufs = static_cast<char *>(ws.batch.p);

    std::vector<StageJob> jobs;
    long long stage_rows = 0;
    WorkList L;
    ImagePlan plan;
    for (int i = 0; i < n; ++i) {
        Img &m = im[i];
        if (m.stage) {
            char *sb = bufs + m.stage_off;
            Input c = m.in;
            c.I = sb;
            c.A = sb + m.stage_offA;
            c.I_pitch = m.pI;
            c.A_pitch = m.pA;
            c.padded = true;
            jobs.push_back(StageJob{m.in.I, sb, m.in.I_pitch * es, m.pI * es, 3LL * m.in.w * es, m.in.h,
                                    stage_rows});
            stage_rows += m.in.h;
            jobs.push_back(StageJob{m.in.A, sb + m.stage_offA, m.in.A_pitch * es, m.pA * es,
                                    (long long)m.in.w * es, m.in.h, stage_rows});
            stage_rows += m.in.h;
            m.in = c;
        }
        if (!plan_image(dtype, p, m.in, m.lv, m.nc, F[i].ptr, B[i].ptr, F[i].row_pitch_bytes / es,
                        bufs + m.buf_off, bufs + m.buf_off + m.need, m.need, plan)) {
            // a 16-bit pass whose rows would need per-lane copies off the 4-byte grid
            for (int k = 0; k < n; ++k)
                if ((st = estimate(im[k].orig, dtype, p, F[k].ptr, B[k].ptr, F[k].row_pitch_bytes / es, s)) != FG_OK)
                    return st;
            return FG_OK;
        }
        worklist_add(L, plan, true, 0, (int)plan.passes.size());
    }
    if ((st = worklist_finish(L)) != FG_OK) return st;
    const WorkListLayout o = worklist_layout(L, jobs.size());
    const std::vector<char> blob = worklist_blob(L, jobs, o);

    // A graph cached for this batch keeps its own copy of the work list (descriptors, items,
    // counters), so that another batch on this stream cannot overwrite it; the levels and
    // staged copies stay in the shared workspace, which runs on this stream one batch at a time.
    Buf own;
    if (!key.empty() && cudaMallocAsync(&own.p, o.bytes, s) == cudaSuccess) {
        own.bytes = o.bytes;
    } else {
        cudaGetLastError();
        own.p = nullptr;
        key.clear();
        if ((st = ensure(ws.worklist, o.bytes, s)) != FG_OK) return st;
    }
    char *wl = static_cast<char *>(own.p ? own.p : ws.worklist.p);
    cudaError_t e = cudaMemcpyAsync(wl, blob.data(), blob.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        if (own.p) cudaFreeAsync(own.p, s);
        return cuda_fail(e, "copy of the batch work list");
    }
    if (key.empty()) return worklist_enqueue(dtype, p.clamp, L, o, jobs.size(), stage_rows, wl, s);
    cudaStream_t cs = capture_stream();
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    if (cs && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        st = worklist_enqueue(dtype, p.clamp, L, o, jobs.size(), stage_rows, wl, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (st == FG_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (!ex) {   // capture unavailable or refused: launch directly from the owned work list
        cudaGetLastError();
        st = worklist_enqueue(dtype, p.clamp, L, o, jobs.size(), stage_rows, wl, s);
        cudaFreeAsync(own.p, s);
        return st;
    }
    evict_graphs(ws, s);
    ws.graphs.emplace(key, ex);
    ws.graph_order.push_back(key);
    ws.graph_bufs.emplace(key, own);
    e = cudaGraphLaunch(ex, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    return FG_OK;
}

extern "C" fg_status fg_autotune_batch(int n, const fg_image *I, const fg_image *alpha,
                                       const fg_params *params, fg_image *F, fg_image *B,
                                       void *stream, int *chosen, float *ms) {
    g_err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    const int nc = (int)(sizeof kStripCandidates / sizeof kStripCandidates[0]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "autotune events");
    }
    BatchStrips keep;
    {
        std::lock_guard<std::mutex> lk(g_strips_mu);
        keep = g_strips;
    }
    int best = -1;
    float best_ms = 0.f;
    fg_status st = FG_OK;
    for (int c = 0; c < nc && st == FG_OK; ++c) {
        {
            std::lock_guard<std::mutex> lk(g_strips_mu);
            g_strips = kStripCandidates[c];
        }
        // two untimed calls (workspace growth; the second captures the batch's graph),
        // then two timed ones
        for (int r = 0; r < 2 && st == FG_OK; ++r) st = fg_estimate_batch(n, I, alpha, params, F, B, stream);
        if (st != FG_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && st == FG_OK; ++r) st = fg_estimate_batch(n, I, alpha, params, F, B, stream);
        if (st != FG_OK) break;
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (best < 0 || t < best_ms) {
            best = c;
            best_ms = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_strips_mu);
        g_strips = st == FG_OK && best >= 0 ? kStripCandidates[best] : keep;
        g_strips_cache_read = true;
    }
    if (st != FG_OK) return st;
    write_tune_cache(kStripCandidates[best]);
    if (chosen) *chosen = best;
    if (ms) *ms = best_ms / 2;
    return FG_OK;
}

extern "C" fg_status fg_selftest_bounded_wait(void *stream) {
    g_err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    Workspace &ws = workspace_for(s);
    const size_t off_item = align256(sizeof(BatchDesc)), off_cnt = off_item + 256;
    if (ws.batch.bytes < off_cnt + 256) {
        cudaStreamSynchronize(s);
        clear_graphs(ws, s);   // cached batch graphs point into the buffer about to be replaced
    }
    fg_status st = ensure(ws.batch, off_cnt + 256, s);
    if (st != FG_OK) return st;
    // one item that waits for its own pass: the count it waits for is never reached
    BatchDesc d;
    std::memset(&d, 0, sizeof d);
    d.iters = 2;
    d.dep = 0;
    d.dep_count = 1;
    BatchItem it{0, 0};
    char *dev = (char *)ws.batch.p;
    std::vector<char> blob(off_cnt + 256, 0);
    std::memcpy(blob.data(), &d, sizeof d);
    std::memcpy(blob.data() + off_item, &it, sizeof it);
    cudaError_t e = cudaMemcpyAsync(dev, blob.data(), blob.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test upload");
    BatchLaunch b;
    b.descs = reinterpret_cast<const BatchDesc *>(dev);
    b.items = reinterpret_cast<const BatchItem *>(dev + off_item);
    b.n_items = 1;
    b.counters = reinterpret_cast<int *>(dev + off_cnt);
    b.wait_ns = 20000000;   // 20 ms
    b.slot_bytes = 0;
    b.region = 128;
    b.blocks = 1;
    e = launch_tile_batch(kF32, 1, b, s, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test synchronize");
    int code = 0;
    e = read_and_clear_device_error(&code, s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test error word");
    if (code != 2) return fail(FG_ERR_CUDA, "the bounded wait did not report a timeout (code %d)", code);
    return fail(FG_ERR_TIMEOUT, "bounded wait gave up as intended");
}

// ====================================================== level-granular serving support

namespace fgml {

struct ServePlan {
    ImagePlan image;
    std::vector<long long> work;   // pixels x sweeps of each pass
};

// Strip shape of serving plans (FGML_SERVE_STRIPS="per_sm,lo,hi" overrides): a launch
// often holds few jobs, so strips are short enough that each level's strips spread over
// the SMs and the level chain of a job is not one warp walking tall strips.
BatchStrips serve_strips() {
    static const BatchStrips v = [] {
        BatchStrips d{16, 4, 64};   // measured: half the single-job latency of {4, 28, 124}
        const char *e = std::getenv("FGML_SERVE_STRIPS");
        int a, b, c;
        if (e && std::sscanf(e, "%d,%d,%d", &a, &b, &c) == 3 && a > 0 && b > 0 && c >= b) d = {a, b, c};
        return d;
    }();
    return v;
}

size_t serve_level_bytes(int w, int h, int dtype, const fg_params &p) {
    const std::vector<Level> lv = plan_levels(w, h, p);
    return image_level_bytes(lv, coarse_levels(lv), dtype == kF32 ? 4 : 2);
}

bool serve_supported(const fg_params &p) {
    return p.order == FG_ORDER_JACOBI && p.small_iters > 0 && p.big_iters > 0;
}

fg_status serve_plan_create(int dtype, const fg_params &p, const void *I, long long I_pitch,
                            const void *A, long long A_pitch, bool padded, int w, int h, void *F,
                            void *B, long long d_pitch, void *lev0, void *lev1, ServePlan **out) {
    g_err.clear();
    const int es = dtype == kF32 ? 4 : 2;
    if (!rows_on_grid(I, I_pitch * es) || !rows_on_grid(A, A_pitch * es))
        return fail(FG_ERR_INVALID_ARG, "serving plans need I and alpha rows on the 16-byte grid");
    Input in{I, A, I_pitch, A_pitch, w, h};
    in.padded = padded;
    const std::vector<Level> lv = plan_levels(w, h, p);
    const int nc = coarse_levels(lv);
    std::unique_ptr<ServePlan> sp(new ServePlan());
    const BatchStrips strips = serve_strips();
    if (!plan_image(dtype, p, in, lv, nc, F, B, d_pitch, lev0, lev1, image_level_bytes(lv, nc, es),
                    sp->image, &strips))
        return fail(FG_ERR_CUDA, "no chunk layout for a %dx%d job", w, h);
    for (const BatchDesc &d : sp->image.passes) sp->work.push_back((long long)d.a.w * d.a.h * d.iters);
    *out = sp.release();
    return FG_OK;
}

void serve_plan_destroy(ServePlan *plan) { delete plan; }

int serve_plan_passes(const ServePlan *plan) { return (int)plan->image.passes.size(); }

long long serve_plan_work(const ServePlan *plan, int j) { return plan->work[j]; }

fg_status serve_reserve(cudaStream_t s, size_t worklist_bytes) {
    return ensure(workspace_for(s).worklist, worklist_bytes, s);
}

fg_status serve_launch(int dtype, const fg_params &p, const ServePart *parts, int n, cudaStream_t s) {
    g_err.clear();
    WorkList L;
    for (int i = 0; i < n; ++i)
        worklist_add(L, parts[i].plan->image, parts[i].coarse != 0, parts[i].first, parts[i].last);
    fg_status st = worklist_finish(L);
    if (st != FG_OK) return st;
    const WorkListLayout o = worklist_layout(L, 0);
    const std::vector<char> blob = worklist_blob(L, {}, o);
    Workspace &ws = workspace_for(s);
    if ((st = ensure(ws.worklist, o.bytes, s)) != FG_OK) return st;
    char *wl = static_cast<char *>(ws.worklist.p);
    cudaError_t e = cudaMemcpyAsync(wl, blob.data(), blob.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the serving work list");
    return worklist_enqueue(dtype, p.clamp, L, o, 0, 0, wl, s);
}

}  // namespace fgml
