// Internal declarations shared by the Splotch CUDA translation units (sm_103a).
//
// The per-particle raster rule lives here as device code: roto-translation and
// perspective projection with the camera and look-at parameters, near-plane clipping,
// screen radius from the smoothing length (Section 2.1), the pixel box, the tile rule
// "distance to tile centre < 0.75 radius + sqrt(2) tile / 2" (Section 3.2.1) and the
// per-pixel coverage of the Gaussian footprint.  Every comparison that decides an
// integer is evaluated with explicitly rounded FP32 operations (no contraction) so the
// decisions are reproducible from the ABI's written rule.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spl {

constexpr int kMaxTiles = 16384;   // tiles per image (per-CTA shared histogram)
constexpr int kMaxTile = 64;       // tile edge in pixels (shared accumulator)
constexpr int kMaxTypes = 255;     // species (8-bit type field in the tile records)
constexpr int kThreads = 1024;     // CTA size of the particle-stream kernels (one per SM: one tile histogram per SM)
constexpr int kSplatThreads = 256; // CTA size of the splat kernel for tiles above 32 px
constexpr int kSplatWarps = kSplatThreads / 32;
constexpr int kStage = 512;        // tile records per bulk-copy stage (tiles above 32 px)
constexpr int kMaxGroup = 16;      // views per CTA in the particle-stream kernels
constexpr uint32_t kCodeMax = 16777215u;   // 24-bit normalised-intensity code
constexpr float kLog2e = 1.4426950408889634f;

// Per-view constants, all FP32 except the integer geometry.
struct ViewParams {
    float m[12];          // 3x4 view matrix (rows s, u, f with translations)
    float F, cx, cy, zn;  // focal length (px), image centre, near plane
    float zf;             // far plane (+infinity when there is none)
    float rfac, rmin;     // support factor and floor
    float kexp;           // -log2(e) / sigma_over_R^2: w = exp2(d2 * kexp / R^2)
    float hd;             // 0.70710677 * T, rounded once
    int W, H, T, ntx, nty, n_tiles;
    uint32_t tmagic;      // floor(2^32 / T) + 1: pixel -> tile index by one multiply-high
    int fastdiv;          // 1 when W, H <= 65536 and T > 1 (the multiply-high is exact there)
};

// Tile index of a pixel coordinate (>= 0): q = floor(p / T).  For p < 2^16 and T <= 64 the
// product p * (floor(2^32 / T) + 1) / 2^32 errs by less than 2^-16 < 1 / T, so the floor is exact.
__device__ __forceinline__ int tile_of(const ViewParams &v, int p) {
    return v.fastdiv ? (int)__umulhi((unsigned)p, v.tmagic) : p / v.T;
}

// Device-resident scene as the kernels see it.
struct SceneDev {
    const void *x, *y, *z, *h, *it;  // SoA in the storage type, padded
    int64_t n;
    int n_types;
    const int64_t *type_begin;       // [n_types + 1]
    const float4 *lut;               // brightness x colormap entries, all species
    const int *lut_off;              // [n_types]
    const int *lut_len;              // [n_types]
    const float4 *emit;              // [n] {r, g, b, species bits}: per-particle emission
                                     // (vector colour scenes; records then carry particle
                                     // indices), or null
};

// Per-frame buffers (one frame = V views).
struct FrameDev {
    const ViewParams *views;  // [V]
    int V, G;                 // views, views per particle-stream CTA
    int n_tiles;              // per view
    int T;                    // tile edge (all views)
    int64_t chunk;            // particles per particle-stream CTA
    int n_chunks;
    int *counts;              // [V * n_tiles]
    int *rel;                 // [V * n_chunks * n_tiles] chunk base inside the tile segment
    int64_t *offsets;         // [V * n_tiles + 1] tile segment starts in `lists`
    int *item_off;            // [V * n_tiles + 1] first work item of each tile
    int *split_slot;          // [V * n_tiles] scratch slot of tiles split over items, else -1
    int64_t *sizes;           // [8] pairs, items, splits, K, max tile count
    int *status;              // [4] 0: capacity overflow, 1: timeout, 2: work queue
    float4 *lists;            // [pair capacity] tile records (X, Y, R, code)
    int *pids;                // [pair capacity] particle index per record, or null
    unsigned long long *scratch;  // [split capacity][3][T][T][2] exact accumulators (fix_add)
    int *tickets;                 // [split capacity]
    int *order;                   // [item capacity] work items, largest first (k_item_order), or
                                  // null: items in tile order
    int64_t pair_cap;
    int item_cap, split_cap;
    const float *vscale;      // [V * n_types] emission scale per view and species, or null
    // per-view colormaps (set with vscale): entries (premultiplied by brightness) of
    // view v, species t at vlut[vlut_off[v * n_types + t] ...], vlut_len[...] of them
    const float4 *vlut;
    const int *vlut_off, *vlut_len;
};

enum { kSizePairs = 0, kSizeItems = 1, kSizeSplits = 2, kSizeK = 3, kSizeMaxCount = 4 };
enum { kStatOverflow = 0, kStatTimeout = 1, kStatQueue = 2 };

// ------------------------------------------------------------------------------------
// Storage loaders: VEC consecutive particles with one 16-byte load per attribute.

template <int S> struct Store;
template <> struct Store<0> {
    static constexpr int VEC = 4;
    static constexpr int BYTES = 4;
    __device__ __forceinline__ static void load(const void *p, int64_t i, float *v) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(p) + i));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};
template <> struct Store<1> {
    static constexpr int VEC = 8;
    static constexpr int BYTES = 2;
    __device__ __forceinline__ static void load(const void *p, int64_t i, float *v) {
        uint4 a = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __half *>(p) + i));
        const __half2 *q = reinterpret_cast<const __half2 *>(&a);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __half22float2(q[k]);
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
};
template <> struct Store<2> {
    static constexpr int VEC = 8;
    static constexpr int BYTES = 2;
    __device__ __forceinline__ static void load(const void *p, int64_t i, float *v) {
        uint4 a = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(p) + i));
        const __nv_bfloat162 *q = reinterpret_cast<const __nv_bfloat162 *>(&a);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(q[k]);
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
};

// One attribute of one particle (a warp reads 32 consecutive particles: coalesced).
template <int S> __device__ __forceinline__ float load1(const void *p, int64_t i);
template <> __device__ __forceinline__ float load1<0>(const void *p, int64_t i) {
    return __ldg(static_cast<const float *>(p) + i);
}
template <> __device__ __forceinline__ float load1<1>(const void *p, int64_t i) {
    return __half2float(__ldg(static_cast<const __half *>(p) + i));
}
template <> __device__ __forceinline__ float load1<2>(const void *p, int64_t i) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(p) + i));
}

// ------------------------------------------------------------------------------------
// Raster rule (FP32, each operation rounded once, left to right).

struct Raster {
    float X, Y, R, zc;
    int i0, i1, j0, j1;
};

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// Returns true when the particle is active: in front of the near plane, finite, and
// with a non-empty pixel box inside the image.
__device__ __forceinline__ bool raster_one(const ViewParams &v, float x, float y, float z, float h,
                                           Raster &o) {
    const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(v.m[0], x), __fmul_rn(v.m[1], y)),
                                         __fmul_rn(v.m[2], z)), v.m[3]);
    const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(v.m[4], x), __fmul_rn(v.m[5], y)),
                                         __fmul_rn(v.m[6], z)), v.m[7]);
    const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(v.m[8], x), __fmul_rn(v.m[9], y)),
                                         __fmul_rn(v.m[10], z)), v.m[11]);
    o.zc = zc;
    if (!(zc > v.zn) || !(zc <= v.zf)) return false;
    const float X = __fadd_rn(v.cx, __fdiv_rn(__fmul_rn(v.F, xc), zc));
    const float Y = __fsub_rn(v.cy, __fdiv_rn(__fmul_rn(v.F, yc), zc));
    const float r = __fdiv_rn(__fmul_rn(v.F, h), zc);
    float R = __fmul_rn(v.rfac, r);
    if (!(R > v.rmin)) R = v.rmin;
    o.X = X; o.Y = Y; o.R = R;
    if (!(isfinite(X) && isfinite(Y) && isfinite(R))) return false;
    const float wmax = (float)v.W + 1.0f, hmax = (float)v.H + 1.0f;
    const float xl = clampf(__fsub_rn(__fsub_rn(X, R), 0.5f), -2.0f, wmax);
    const float xh = clampf(__fsub_rn(__fadd_rn(X, R), 0.5f), -2.0f, wmax);
    const float yl = clampf(__fsub_rn(__fsub_rn(Y, R), 0.5f), -2.0f, hmax);
    const float yh = clampf(__fsub_rn(__fadd_rn(Y, R), 0.5f), -2.0f, hmax);
    o.i0 = max(0, (int)ceilf(xl) - 1);
    o.i1 = min(v.W - 1, (int)floorf(xh) + 1);
    o.j0 = max(0, (int)ceilf(yl) - 1);
    o.j1 = min(v.H - 1, (int)floorf(yh) + 1);
    return o.i0 <= o.i1 && o.j0 <= o.j1;
}

// Box of a particle already rasterised (X, Y, R known): same expressions as above.
__device__ __forceinline__ void pixel_box(const ViewParams &v, float X, float Y, float R, int &i0,
                                          int &i1, int &j0, int &j1) {
    const float wmax = (float)v.W + 1.0f, hmax = (float)v.H + 1.0f;
    i0 = max(0, (int)ceilf(clampf(__fsub_rn(__fsub_rn(X, R), 0.5f), -2.0f, wmax)) - 1);
    i1 = min(v.W - 1, (int)floorf(clampf(__fsub_rn(__fadd_rn(X, R), 0.5f), -2.0f, wmax)) + 1);
    j0 = max(0, (int)ceilf(clampf(__fsub_rn(__fsub_rn(Y, R), 0.5f), -2.0f, hmax)) - 1);
    j1 = min(v.H - 1, (int)floorf(clampf(__fsub_rn(__fadd_rn(Y, R), 0.5f), -2.0f, hmax)) + 1);
}

// Tile rule of Section 3.2.1 with the clamped support R standing for 0.75 radius.
__device__ __forceinline__ bool tile_member(const ViewParams &v, float X, float Y, float R, int tx,
                                            int ty) {
    const float T = (float)v.T;
    const float cx = __fmul_rn(__fadd_rn((float)tx, 0.5f), T);
    const float cy = __fmul_rn(__fadd_rn((float)ty, 0.5f), T);
    const float ex = __fsub_rn(cx, X), ey = __fsub_rn(cy, Y);
    const float q = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
    const float thr = __fadd_rn(R, v.hd);
    return q < __fmul_rn(thr, thr);
}

// Lanes of the (full) warp whose key equals this lane's in the low NB bits, found bit by
// bit with ballots: NB ballots, independent of how many distinct keys the warp holds.
template <int NB> __device__ __forceinline__ uint32_t warp_peers(uint32_t key) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < NB; ++bit) {
        const uint32_t on = (key >> bit) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, on);
        peers &= on ? bal : ~bal;
    }
    return peers;
}

// Inclusive warp scan of an int.
__device__ __forceinline__ int warp_incl_scan_i(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// ------------------------------------------------------------------------------------
// Bulk-copy (TMA, non-tensor) and mbarrier helpers.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Plain arrival (release semantics at CTA scope: this thread's earlier shared-memory
// writes are visible to a thread whose wait observes the phase completing).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of a phase's completion.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~`limit` SM cycles and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------------------------------------
// Exact, order-independent merge of FP32 partial sums (slices of a split tile).  A value
// is taken as a signed 128-bit integer count of 2^-64 (magnitudes below 2^-64 drop out,
// magnitudes from 2^62 up saturate there) and added to a {low, high} pair of 64-bit words
// with two integer atomics, the low word's carry going into the high one.  Integer
// addition is associative, so the merged sum is the same whichever slice arrives first;
// fix_value rounds it to FP32 once.

__device__ __forceinline__ void fix_add(unsigned long long *acc, float v) {
    const uint32_t b = __float_as_uint(v);
    const int E = (int)((b >> 23) & 0xFFu);
    if (E == 0) return;  // zero or subnormal: below the unit
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = E - 86;  // |v| * 2^64 = m * 2^(E - 150 + 64)
    unsigned long long lo, hi;
    if (sh <= -24) return;
    if (sh < 0) lo = m >> (-sh), hi = 0ull;
    else if (sh == 0) lo = m, hi = 0ull;
    else if (sh < 64) lo = m << sh, hi = m >> (64 - sh);
    else if (sh < 102) lo = 0ull, hi = m << (sh - 64);
    else lo = 0ull, hi = 1ull << 62;
    if (b >> 31) {  // two's complement of the 128-bit magnitude
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const unsigned long long old = atomicAdd(&acc[0], lo);
    const unsigned long long up = hi + (old + lo < old ? 1ull : 0ull);
    if (up) atomicAdd(&acc[1], up);
}

// Value of an accumulator pair once every addition into it is complete and visible.
__device__ __forceinline__ float fix_value(const unsigned long long *acc) {
    const unsigned long long lo = __ldcg(&acc[0]), hi = __ldcg(&acc[1]);
    const double d = (double)(long long)hi * 18446744073709551616.0 + (double)lo;
    return (float)(d * 5.4210108624275222e-20);  // x 2^-64
}

// 2^x on the SFU (PTX ex2.approx.ftz, max relative error about 2^-22); the weights it feeds
// are values, never decisions.
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------------------------
// Host-side launchers (defined in the kernel translation units).

cudaError_t launch_minmax(int storage_in_f32_only, const float *I, int64_t begin, int64_t end, int i_log,
                          unsigned *keys, cudaStream_t st);
cudaError_t launch_emission(int storage, const SceneDev &sc, const float *rgb, const int *vec, const float *lo,
                            const float *hi, const int *lg, const float *beta, float4 *emit, int *bad,
                            cudaStream_t st);
cudaError_t launch_prepare(const float *x, const float *y, const float *z, const float *h,
                           const float *I, int64_t n, int n_types, const int64_t *type_begin,
                           const float *lo, const float *hi, const int *i_log, int storage,
                           void *ox, void *oy, void *oz, void *oh, void *oit, int *bad,
                           cudaStream_t st);
cudaError_t launch_count(int storage, const SceneDev &sc, const FrameDev &fr, cudaStream_t st);
cudaError_t launch_scan(const FrameDev &fr, int target_items, int kmin, cudaStream_t st);
// stable: every tile list in ascending particle index (k_scatter_stable); else each
// chunk's members in arrival order (k_scatter)
cudaError_t launch_scatter(int storage, const SceneDev &sc, const FrameDev &fr, bool stable, cudaStream_t st);
cudaError_t launch_splat(const SceneDev &sc, const FrameDev &fr, int *queue, float *out,
                         int out_accum, int grid, cudaStream_t st);
int splat_blocks_per_sm(int T);
int splat_workers_per_sm(int T);
int splat_split(int T);  // squares per tile edge the splat renders separately (1 or 2)
int bin_ctas_per_sm(int storage, size_t smem);

// Raise a kernel's dynamic shared-memory limit on the current device to at least
// `bytes`, once per (kernel, device).  The limit is process-wide state: renders on other
// host threads launch the same kernels, so it is only ever raised, never set per launch.
cudaError_t ensure_smem_limit(const void *kernel, size_t bytes);

// Stable LSD radix sort of (64- or 32-bit key, 32-bit value) pairs by key bits
// [bit_lo, bit_hi) (8 bits per pass); the result is in the alternate buffers when *in_alt.
size_t sort_temp_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int bit_lo, int bit_hi, void *temp, cudaStream_t st, bool *in_alt);
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int bit_lo, int bit_hi, void *temp, cudaStream_t st, bool *in_alt);
// Sort by key bits [bit_lo, bit_hi) whose values index `payload`, and write the payload in
// sorted order to payload_out (the last pass gathers; keys and values end up undefined).
cudaError_t radix_sort_gather(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                              int bit_lo, int bit_hi, void *temp, const float4 *payload, float4 *payload_out,
                              cudaStream_t st);
// In-place exclusive scan of 32-bit counts whose total stays below 2^32.
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan_u32(uint32_t *a, int64_t n, void *temp, cudaStream_t st);

// Depth-ordered binning of one view (views[0]): per-particle records and depth keys (with
// the range of the active keys, and their rebasing to it), the
// counts in sorted order (cnt has n + 1 entries, the last set to 0), and the expansion
// into (tile id, slot) pairs at the scanned offsets; k_expand flags kStatOverflow in
// `status` if a particle's tiles disagree with its count.
cudaError_t launch_depth_records(int storage, const SceneDev &sc, const ViewParams *views, float4 *prec,
                                 uint32_t *dkey, uint32_t *pid, uint32_t *krange, cudaStream_t st);
cudaError_t launch_rebase_keys(uint32_t *dkey, int64_t n, uint32_t base, uint32_t span, cudaStream_t st);
cudaError_t launch_sorted_counts(const ViewParams *views, const float4 *prec, const uint32_t *skey,
                                 const uint32_t *spid, int64_t n, uint32_t inactive, float4 *srec, uint32_t *cnt,
                                 cudaStream_t st);
cudaError_t launch_expand(const ViewParams *views, const float4 *srec, const uint32_t *poff, int64_t n, int64_t P,
                          float4 *recs, uint32_t *tkey, uint32_t *tval, int *status, cudaStream_t st);

// Depth-ordered render: record gather by sorted index and the ordered splat (tiles up to
// 32 px; squares of up to 16 px, split when T > 16).
cudaError_t launch_gather_records(const float4 *src, const uint32_t *idx, int64_t n, float4 *dst, cudaStream_t st);
int ordered_split(int T);
int ordered_ctas_per_sm();
int ordered_workers_per_sm();
// Work items of the frame ordered largest first into fr.order (k_item_order; no-op when
// fr.order is null).
cudaError_t launch_item_order(const FrameDev &fr, cudaStream_t st);
cudaError_t launch_splat_ordered(const SceneDev &sc, const FrameDev &fr, int *queue, float *out,
                                 const float *absorb, float *ord_scratch, int map_out, int grid, cudaStream_t st);
size_t splat_smem_bytes(int T);
cudaError_t launch_selftest_wait(long long limit, int *result, cudaStream_t st);
cudaError_t launch_final(float *a, int64_t count, cudaStream_t st);
cudaError_t launch_compose_maps(const float *maps, int n, int64_t pixels, float *out, cudaStream_t st);
cudaError_t launch_debug_raster(int storage, const SceneDev &sc, const ViewParams *view,
                                float *out8, cudaStream_t st);

}  // namespace spl
