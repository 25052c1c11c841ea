// Scene preparation and tile binning (count / scan / scatter) for the Splotch hot path.
//
// Section 3.1 builds, per tile, the list of particles that affect it; Section 3.2.1
// gives the membership rule and notes that growing per-thread vectors stalled on
// allocation.  Here the lists are one flat array sized exactly from a counting pass:
//   k_count      streams the particles once (coalesced SoA loads), rasterises them
//                for a group of views, histograms tile memberships in shared memory and
//                writes each chunk's count of every tile;
//   k_chunk_scan scans every tile's counts over the chunks in chunk order: the base of
//                each chunk's slice of the tile segment, and the tile's total;
//   k_scan       turns the totals into tile segment offsets and the splat's work items;
//   k_scatter    streams the particles again and writes a 16-byte record per
//                (particle, tile) pair into its tile segment (each chunk's slice in the
//                order its warps reach the records); k_scatter_stable writes every slice
//                in ascending particle index, as Section 3.2.1 builds the lists by walking
//                the particles in order.
#include "splotch_internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

namespace spl {

cudaError_t ensure_smem_limit(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[std::make_pair(kernel, dev)];
    if (cur >= bytes) return cudaSuccess;
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    // the largest shared-memory carveout, so that the CTAs the occupancy allows all fit
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err == cudaSuccess) cur = bytes;
    return err;
}

// largest tile histogram: G x n_tiles <= kMaxTiles counters
constexpr size_t kBinSmemMax = sizeof(int) * (size_t)kMaxTiles;


// ---------------------------------------------------------------------------------------
// Scene preparation (Section 2.1: ranging, normalisation, optional logarithm).

__device__ __forceinline__ unsigned order_key(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Sort key of a depth z_c such that ascending keys run from the farthest particle to the
// nearest: the order-preserving unsigned image of the float, complemented.
__device__ __forceinline__ uint32_t depth_key(float zc) { return ~order_key(zc); }
constexpr uint32_t kInactiveKey = 0xFFFFFFFFu;  // no finite depth in front of the near plane maps here

__global__ void k_minmax(const float *__restrict__ I, int64_t begin, int64_t end, int i_log,
                         unsigned *keys) {
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = I[i];
        if (i_log) v = logf(fmaxf(v, 1e-30f));
        if (!isfinite(v)) continue;
        unsigned k = order_key(v);
        lo = min(lo, k);
        hi = max(hi, k);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&keys[0], lo);
        atomicMax(&keys[1], hi);
    }
}

cudaError_t launch_minmax(int, const float *I, int64_t begin, int64_t end, int i_log, unsigned *keys,
                          cudaStream_t st) {
    if (end <= begin) return cudaSuccess;
    int64_t blocks = (end - begin + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_minmax<<<(int)blocks, 256, 0, st>>>(I, begin, end, i_log, keys);
    return cudaGetLastError();
}

template <typename T> __device__ __forceinline__ T to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

template <typename T>
__global__ void k_prepare(const float *__restrict__ x, const float *__restrict__ y,
                          const float *__restrict__ z, const float *__restrict__ h,
                          const float *__restrict__ I, int64_t n, int n_types,
                          const int64_t *__restrict__ tb, const float *__restrict__ lo,
                          const float *__restrict__ hi, const int *__restrict__ i_log, T *ox, T *oy,
                          T *oz, T *oh, T *oit, int *bad, int64_t first) {
    for (int64_t i = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int a = 0, b = n_types - 1;  // species: last t with tb[t] <= i
        while (a < b) {
            int mid = (a + b + 1) >> 1;
            if (tb[mid] <= i) a = mid; else b = mid - 1;
        }
        const float xv = x[i], yv = y[i], zv = z[i], hv = h[i], Iv = I[i];
        if (!(isfinite(xv) && isfinite(yv) && isfinite(zv) && isfinite(hv) && hv > 0.0f && isfinite(Iv)))
            atomicOr(bad, 1);
        float v = i_log[a] ? logf(fmaxf(Iv, 1e-30f)) : Iv;
        const float span = __fsub_rn(hi[a], lo[a]);
        float t = span > 0.0f ? __fdiv_rn(__fsub_rn(v, lo[a]), span) : 0.0f;
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        ox[i] = to_store<T>(xv);
        oy[i] = to_store<T>(yv);
        oz[i] = to_store<T>(zv);
        oh[i] = to_store<T>(hv);
        oit[i] = to_store<T>(t);
    }
}

// Four consecutive particles per thread with 16-byte loads of every input array (inputs
// 16-byte aligned): a quarter of the memory requests, which matters when the inputs are
// read in place from page-locked host memory over the host link.
template <typename T>
__global__ void k_prepare4(const float4 *__restrict__ x, const float4 *__restrict__ y,
                           const float4 *__restrict__ z, const float4 *__restrict__ h,
                           const float4 *__restrict__ I, int64_t n4, int n_types,
                           const int64_t *__restrict__ tb, const float *__restrict__ lo,
                           const float *__restrict__ hi, const int *__restrict__ i_log, T *ox, T *oy,
                           T *oz, T *oh, T *oit, int *bad) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        const float4 xv = x[q], yv = y[q], zv = z[q], hv = h[q], Iv = I[q];
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w}, ys[4] = {yv.x, yv.y, yv.z, yv.w};
        const float zs[4] = {zv.x, zv.y, zv.z, zv.w}, hs[4] = {hv.x, hv.y, hv.z, hv.w};
        const float is[4] = {Iv.x, Iv.y, Iv.z, Iv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = 4 * q + k;
            int a = 0, b = n_types - 1;  // species: last t with tb[t] <= i
            while (a < b) {
                int mid = (a + b + 1) >> 1;
                if (tb[mid] <= i) a = mid; else b = mid - 1;
            }
            if (!(isfinite(xs[k]) && isfinite(ys[k]) && isfinite(zs[k]) && isfinite(hs[k]) && hs[k] > 0.0f &&
                  isfinite(is[k])))
                atomicOr(bad, 1);
            float v = i_log[a] ? logf(fmaxf(is[k], 1e-30f)) : is[k];
            const float span = __fsub_rn(hi[a], lo[a]);
            float t = span > 0.0f ? __fdiv_rn(__fsub_rn(v, lo[a]), span) : 0.0f;
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            ox[i] = to_store<T>(xs[k]);
            oy[i] = to_store<T>(ys[k]);
            oz[i] = to_store<T>(zs[k]);
            oh[i] = to_store<T>(hs[k]);
            oit[i] = to_store<T>(t);
        }
    }
}

template <typename T>
static void prepare_launch(const float *x, const float *y, const float *z, const float *h, const float *I,
                           int64_t n, int n_types, const int64_t *tb, const float *lo, const float *hi,
                           const int *i_log, void *ox, void *oy, void *oz, void *oh, void *oit, int *bad,
                           cudaStream_t st) {
    auto aligned = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    int64_t done = 0;
    if (aligned(x) && aligned(y) && aligned(z) && aligned(h) && aligned(I) && n >= 4) {
        const int64_t n4 = n / 4;
        int64_t blocks = (n4 + 255) / 256;
        if (blocks > 65536) blocks = 65536;
        k_prepare4<T><<<(int)blocks, 256, 0, st>>>((const float4 *)x, (const float4 *)y, (const float4 *)z,
                                                   (const float4 *)h, (const float4 *)I, n4, n_types, tb, lo, hi,
                                                   i_log, (T *)ox, (T *)oy, (T *)oz, (T *)oh, (T *)oit, bad);
        done = 4 * n4;
    }
    if (done < n) {
        // the remaining particles (or all, for unaligned inputs), one per thread; the
        // outputs are offset so indices stay global
        int64_t blocks = (n - done + 255) / 256;
        if (blocks > 65536) blocks = 65536;
        k_prepare<T><<<(int)blocks, 256, 0, st>>>(x, y, z, h, I, n, n_types, tb, lo, hi, i_log, (T *)ox, (T *)oy,
                                                  (T *)oz, (T *)oh, (T *)oit, bad, done);
    }
}

// Per-particle emission of a scene with vector-coloured species (Section 2.1: colour
// directly from a vector input field, or from a scalar through the colormap): for a
// vector species, C~ = clamp((C' - lo) / (hi - lo), 0, 1) per component (C' = ln(max(C,
// 1e-30)) with the log flag; 0 when hi <= lo) and e = brightness C~; for the others the
// colormap (premultiplied by brightness) interpolated at the stored normalised intensity.
// The species index rides in .w.  A non-finite colour component sets *bad.
template <int S>
__global__ void k_emission(SceneDev sc, const float *__restrict__ rgb, const int *__restrict__ vec,
                           const float *__restrict__ lo, const float *__restrict__ hi, const int *__restrict__ lg,
                           const float *__restrict__ beta, float4 *emit, int *bad) {
    __shared__ int64_t s_tb[kMaxTypes + 1];
    for (int k = threadIdx.x; k <= sc.n_types; k += blockDim.x) s_tb[k] = sc.type_begin[k];
    __syncthreads();
    int type = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sc.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        while (type + 1 < sc.n_types && i >= s_tb[type + 1]) ++type;
        float e[3];
        if (vec[type]) {
            const float l = lo[type], span = hi[type] - l;
            for (int c = 0; c < 3; ++c) {
                float v = rgb[3 * i + c];
                if (!isfinite(v)) atomicExch(bad, 1);
                if (lg[type]) v = logf(fmaxf(v, 1e-30f));
                float t = span > 0.0f ? (v - l) / span : 0.0f;
                t = fminf(fmaxf(t, 0.0f), 1.0f);
                e[c] = beta[type] * t;
            }
        } else {
            const float It = load1<S>(sc.it, i);
            const int len = sc.lut_len[type];
            const float f = It * (float)(len - 1);
            const int kk = min((int)f, len - 2);
            const float tau = f - (float)kk;
            const float4 c0 = sc.lut[sc.lut_off[type] + kk], c1 = sc.lut[sc.lut_off[type] + kk + 1];
            e[0] = (1.0f - tau) * c0.x + tau * c1.x;
            e[1] = (1.0f - tau) * c0.y + tau * c1.y;
            e[2] = (1.0f - tau) * c0.z + tau * c1.z;
        }
        emit[i] = make_float4(e[0], e[1], e[2], __int_as_float(type));
    }
}

cudaError_t launch_emission(int storage, const SceneDev &sc, const float *rgb, const int *vec, const float *lo,
                            const float *hi, const int *lg, const float *beta, float4 *emit, int *bad,
                            cudaStream_t st) {
    if (sc.n <= 0) return cudaSuccess;
    int64_t blocks = (sc.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (storage == 0) k_emission<0><<<(int)blocks, 256, 0, st>>>(sc, rgb, vec, lo, hi, lg, beta, emit, bad);
    else if (storage == 1) k_emission<1><<<(int)blocks, 256, 0, st>>>(sc, rgb, vec, lo, hi, lg, beta, emit, bad);
    else k_emission<2><<<(int)blocks, 256, 0, st>>>(sc, rgb, vec, lo, hi, lg, beta, emit, bad);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const float *x, const float *y, const float *z, const float *h,
                           const float *I, int64_t n, int n_types, const int64_t *type_begin,
                           const float *lo, const float *hi, const int *i_log, int storage,
                           void *ox, void *oy, void *oz, void *oh, void *oit, int *bad,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    switch (storage) {
    case 0:
        prepare_launch<float>(x, y, z, h, I, n, n_types, type_begin, lo, hi, i_log, ox, oy, oz, oh, oit, bad, st);
        break;
    case 1:
        prepare_launch<__half>(x, y, z, h, I, n, n_types, type_begin, lo, hi, i_log, ox, oy, oz, oh, oit, bad, st);
        break;
    default:
        prepare_launch<__nv_bfloat16>(x, y, z, h, I, n, n_types, type_begin, lo, hi, i_log, ox, oy, oz, oh, oit,
                                      bad, st);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// k_count: raster a chunk of particles for up to G views and count tile memberships.

// Bin one particle for every view of the group: 2 x 2 candidate tiles or fewer by this
// lane, larger candidate boxes by the whole warp (one such particle at a time).  Called by
// all lanes of the warp together.
__device__ __forceinline__ void count_particle(bool valid, float x, float y, float z, float h,
                                               const ViewParams *s_view, int g_n, int *s_hist, int nt,
                                               int lane) {
    for (int g = 0; g < g_n; ++g) {
        const ViewParams &vp = s_view[g];
        int *hist = s_hist + g * nt;
        Raster r;
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (valid && raster_one(vp, x, y, z, h, r)) {
            tx0 = tile_of(vp, r.i0), tx1 = tile_of(vp, r.i1);
            ty0 = tile_of(vp, r.j0), ty1 = tile_of(vp, r.j1);
        }
        const bool small = tx1 >= tx0 && tx1 - tx0 <= 1 && ty1 - ty0 <= 1;
        if (small) {
            const bool m00 = tile_member(vp, r.X, r.Y, r.R, tx0, ty0);
            const bool m10 = tx1 > tx0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty0);
            const bool m01 = ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx0, ty1);
            const bool m11 = tx1 > tx0 && ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty1);
            const int t00 = ty0 * vp.ntx + tx0;
            if (m00) atomicAdd(&hist[t00], 1);
            if (m10) atomicAdd(&hist[t00 + 1], 1);
            if (m01) atomicAdd(&hist[t00 + vp.ntx], 1);
            if (m11) atomicAdd(&hist[t00 + vp.ntx + 1], 1);
        }
        uint32_t big = __ballot_sync(0xffffffffu, tx1 >= tx0 && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const float bX = __shfl_sync(0xffffffffu, r.X, src), bY = __shfl_sync(0xffffffffu, r.Y, src);
            const float bR = __shfl_sync(0xffffffffu, r.R, src);
            const int bx0 = __shfl_sync(0xffffffffu, tx0, src), bx1 = __shfl_sync(0xffffffffu, tx1, src);
            const int by0 = __shfl_sync(0xffffffffu, ty0, src), by1 = __shfl_sync(0xffffffffu, ty1, src);
            const int bw = bx1 - bx0 + 1, ncand = bw * (by1 - by0 + 1);
            for (int k = lane; k < ncand; k += 32) {
                const int ty = by0 + k / bw, tx = bx0 + k % bw;
                if (tile_member(vp, bX, bY, bR, tx, ty)) atomicAdd(&hist[ty * vp.ntx + tx], 1);
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kThreads) k_count(SceneDev sc, FrameDev fr) {
    extern __shared__ int s_hist[];  // [g_n][n_tiles]
    __shared__ ViewParams s_view[kMaxGroup];
    const int b = blockIdx.x;
    const int v0 = blockIdx.y * fr.G;
    const int g_n = min(fr.G, fr.V - v0);
    const int nt = fr.n_tiles;
    for (int k = threadIdx.x; k < g_n * nt; k += blockDim.x) s_hist[k] = 0;
    if (threadIdx.x < g_n) s_view[threadIdx.x] = fr.views[v0 + threadIdx.x];
    __syncthreads();

    const int64_t s = (int64_t)b * fr.chunk;
    const int64_t e = min(sc.n, s + fr.chunk);
    // Two particles per thread per iteration, A and B, each in its own registers: A's next
    // attributes are loaded as soon as A is binned and stay in flight while B is binned
    // (and the other way round), hiding DRAM latency.  The loop runs warp-uniformly (a lane
    // past the chunk end idles) because large particles are binned by the whole warp.
    const int lane = threadIdx.x & 31;
    const int64_t stride = blockDim.x;
    int64_t i = s + threadIdx.x;
    float ax = 0.0f, ay = 0.0f, az = 0.0f, ah = 0.0f, bx = 0.0f, by = 0.0f, bz = 0.0f, bh = 0.0f;
    if (i < e) ax = load1<S>(sc.x, i), ay = load1<S>(sc.y, i), az = load1<S>(sc.z, i), ah = load1<S>(sc.h, i);
    if (i + stride < e)
        bx = load1<S>(sc.x, i + stride), by = load1<S>(sc.y, i + stride), bz = load1<S>(sc.z, i + stride),
        bh = load1<S>(sc.h, i + stride);
    for (; i - lane < e; i += 2 * stride) {
        count_particle(i < e, ax, ay, az, ah, s_view, g_n, s_hist, nt, lane);
        const int64_t ia = i + 2 * stride;
        if (ia < e) ax = load1<S>(sc.x, ia), ay = load1<S>(sc.y, ia), az = load1<S>(sc.z, ia), ah = load1<S>(sc.h, ia);
        if (i + stride - lane >= e) break;
        count_particle(i + stride < e, bx, by, bz, bh, s_view, g_n, s_hist, nt, lane);
        const int64_t ib = i + 3 * stride;
        if (ib < e) bx = load1<S>(sc.x, ib), by = load1<S>(sc.y, ib), bz = load1<S>(sc.z, ib), bh = load1<S>(sc.h, ib);
    }
    __syncthreads();
    // this chunk's count of every tile (zeros included): k_chunk_scan turns the column of
    // each tile into chunk bases in chunk order
    for (int k = threadIdx.x; k < g_n * nt; k += blockDim.x) {
        const int g = k / nt, t = k - g * nt;
        fr.rel[((int64_t)(v0 + g) * fr.n_chunks + b) * nt + t] = s_hist[k];
    }
}

template <int S> static cudaError_t count_impl(const SceneDev &sc, const FrameDev &fr, cudaStream_t st) {
    const size_t smem = (size_t)fr.G * fr.n_tiles * sizeof(int);
    cudaError_t err = ensure_smem_limit((const void *)k_count<S>, kBinSmemMax);
    if (err != cudaSuccess) return err;
    dim3 grid(fr.n_chunks, (fr.V + fr.G - 1) / fr.G);
    k_count<S><<<grid, kThreads, smem, st>>>(sc, fr);
    return cudaGetLastError();
}

cudaError_t launch_count(int storage, const SceneDev &sc, const FrameDev &fr, cudaStream_t st) {
    if (storage == 0) return count_impl<0>(sc, fr, st);
    if (storage == 1) return count_impl<1>(sc, fr, st);
    return count_impl<2>(sc, fr, st);
}

// ---------------------------------------------------------------------------------------
// k_scan: one CTA.  Tile segment offsets (int64), work items (a tile with more than K
// pairs is split into ceil(count / K) items) and scratch slots of split tiles.

template <typename T> __device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive block scan (1024 threads); returns the exclusive prefix, *total = block sum.
template <typename T> __device__ T block_excl_scan(T v, T *s_warp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = s_warp[lane];
        T wi = warp_incl_scan(w);
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    T res = s_warp[warp] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------------------
// k_chunk_scan: per (view, tile), the exclusive scan of the chunks' counts in chunk order
// (rel becomes each chunk's base inside the tile segment) and the tile's total.  The
// bases depend only on the counts, so the lists' layout is the same on every run.

constexpr int kChunkScanUnroll = 8;

__global__ void __launch_bounds__(256) k_chunk_scan(FrameDev fr) {
    const int nt = fr.n_tiles;
    const int64_t N = (int64_t)fr.V * nt;
    const int nch = fr.n_chunks;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(k / nt), t = (int)(k - (int64_t)v * nt);
        int *col = fr.rel + (int64_t)v * nch * nt + t;
        long long run = 0;
        int b = 0;
        for (; b + kChunkScanUnroll <= nch; b += kChunkScanUnroll) {
            int c[kChunkScanUnroll];
#pragma unroll
            for (int q = 0; q < kChunkScanUnroll; ++q) c[q] = col[(int64_t)(b + q) * nt];
#pragma unroll
            for (int q = 0; q < kChunkScanUnroll; ++q) {
                col[(int64_t)(b + q) * nt] = (int)run;
                run += c[q];
            }
        }
        for (; b < nch; ++b) {
            const int c = col[(int64_t)b * nt];
            col[(int64_t)b * nt] = (int)run;
            run += c;
        }
        // a tile holding 2^31 pairs or more cannot be indexed by the 32-bit cursors
        if (run > (long long)INT32_MAX) {
            atomicExch(&fr.status[kStatOverflow], 1);
            run = INT32_MAX;
        }
        fr.counts[k] = (int)run;
    }
}

constexpr int kScanItems = 4;

__global__ void __launch_bounds__(1024) k_scan(FrameDev fr, int target_items, int kmin) {
    __shared__ long long s_l[33];
    __shared__ int s_i[33];
    __shared__ int s_j[33];
    const int N = fr.V * fr.n_tiles;
    // pass 1: total pairs and largest tile
    long long sum = 0;
    int mx = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int c = fr.counts[k];
        sum += c;
        mx = max(mx, c);
    }
    long long tot;
    block_excl_scan<long long>(sum, s_l, &tot);
    int mx_all;
    {
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) s_i[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = s_i[threadIdx.x];
            for (int o = 16; o; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
            if (threadIdx.x == 0) s_i[32] = w;
        }
        __syncthreads();
        mx_all = s_i[32];
        __syncthreads();
    }
    long long K = (tot + target_items - 1) / (target_items > 0 ? target_items : 1);
    if (K < kmin) K = kmin;
    if (K > (1LL << 30)) K = (1LL << 30);

    // pass 2: scans
    long long run_p = 0;
    int run_i = 0, run_s = 0;
    for (int base = 0; base < N; base += blockDim.x * kScanItems) {
        const int k0 = base + threadIdx.x * kScanItems;
        int c[kScanItems], it[kScanItems], sp[kScanItems];
        long long lp = 0;
        int li = 0, ls = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const int k = k0 + q;
            c[q] = k < N ? fr.counts[k] : 0;
            it[q] = k < N ? max(1, (int)((c[q] + K - 1) / K)) : 0;
            sp[q] = (k < N && c[q] > K) ? 1 : 0;
            lp += c[q];
            li += it[q];
            ls += sp[q];
        }
        long long tp;
        int ti, ts;
        long long ep = block_excl_scan<long long>(lp, s_l, &tp) + run_p;
        int ei = block_excl_scan<int>(li, s_i, &ti) + run_i;
        int es = block_excl_scan<int>(ls, s_j, &ts) + run_s;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const int k = k0 + q;
            if (k < N) {
                fr.offsets[k] = ep;
                fr.item_off[k] = ei;
                fr.split_slot[k] = sp[q] ? es : -1;
            }
            ep += c[q];
            ei += it[q];
            es += sp[q];
        }
        run_p += tp;
        run_i += ti;
        run_s += ts;
    }
    __syncthreads();
    // per-view segment sizes must fit the scatter's 32-bit cursors
    int big = 0;
    for (int v = threadIdx.x; v < fr.V; v += blockDim.x)
        big |= (fr.offsets[(int64_t)v * fr.n_tiles + fr.n_tiles - 1] + fr.counts[(int64_t)v * fr.n_tiles + fr.n_tiles - 1] -
                fr.offsets[(int64_t)v * fr.n_tiles]) > (long long)INT32_MAX;
    big = __syncthreads_or(big);
    if (threadIdx.x == 0) {
        fr.offsets[N] = run_p;
        fr.item_off[N] = run_i;
        fr.sizes[kSizePairs] = run_p;
        fr.sizes[kSizeItems] = run_i;
        fr.sizes[kSizeSplits] = run_s;
        fr.sizes[kSizeK] = K;
        fr.sizes[kSizeMaxCount] = mx_all;
        const bool over = run_p > fr.pair_cap || run_i > fr.item_cap || run_s > fr.split_cap || big ||
                          fr.status[kStatOverflow];
        fr.status[kStatOverflow] = over ? 1 : 0;
    }
}

cudaError_t launch_scan(const FrameDev &fr, int target_items, int kmin, cudaStream_t st) {
    const int64_t N = (int64_t)fr.V * fr.n_tiles;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8192));
    k_chunk_scan<<<blocks, 256, 0, st>>>(fr);
    k_scan<<<1, 1024, 0, st>>>(fr, target_items, kmin);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// k_scatter: same chunks as k_count; every (particle, tile) pair becomes a record
// {X, Y, R, type << 24 | 24-bit normalised intensity} in its tile segment (in scenes with
// a per-particle emission the last word is the particle index).  Each chunk fills its
// slice of a tile segment (slices in chunk order, k_chunk_scan) through a shared-memory
// cursor per tile: the slice holds exactly the chunk's members of the tile, in the order
// the CTA's warps reached them.  k_scatter_stable (below) orders them by particle index.

// Write the records of one particle for every view of the group (same split between
// lane and warp as count_particle).  Called by all lanes of the warp together.
__device__ __forceinline__ void scatter_particle(bool valid, int64_t i, float x, float y, float z, float h,
                                                 float code, const ViewParams *s_view, const int64_t *s_vbase,
                                                 int g_n, int *s_cur, int nt, const FrameDev &fr, int lane) {
    for (int g = 0; g < g_n; ++g) {
        const ViewParams &vp = s_view[g];
        int *cur = s_cur + g * nt;
        float4 *lists = fr.lists + s_vbase[g];
        int *pids = fr.pids ? fr.pids + s_vbase[g] : nullptr;
        Raster r;
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (valid && raster_one(vp, x, y, z, h, r)) {
            tx0 = tile_of(vp, r.i0), tx1 = tile_of(vp, r.i1);
            ty0 = tile_of(vp, r.j0), ty1 = tile_of(vp, r.j1);
        }
        const bool small = tx1 >= tx0 && tx1 - tx0 <= 1 && ty1 - ty0 <= 1;
        if (small) {
            // all cursor reservations first, then the stores: one atomic latency per
            // particle instead of one per tile
            const float4 rec = make_float4(r.X, r.Y, r.R, code);
            const int t00 = ty0 * vp.ntx + tx0;
            const bool m00 = tile_member(vp, r.X, r.Y, r.R, tx0, ty0);
            const bool m10 = tx1 > tx0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty0);
            const bool m01 = ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx0, ty1);
            const bool m11 = tx1 > tx0 && ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty1);
            const int p00 = m00 ? atomicAdd(&cur[t00], 1) : 0;
            const int p10 = m10 ? atomicAdd(&cur[t00 + 1], 1) : 0;
            const int p01 = m01 ? atomicAdd(&cur[t00 + vp.ntx], 1) : 0;
            const int p11 = m11 ? atomicAdd(&cur[t00 + vp.ntx + 1], 1) : 0;
            if (m00) lists[p00] = rec;
            if (m10) lists[p10] = rec;
            if (m01) lists[p01] = rec;
            if (m11) lists[p11] = rec;
            if (pids) {
                if (m00) pids[p00] = (int)i;
                if (m10) pids[p10] = (int)i;
                if (m01) pids[p01] = (int)i;
                if (m11) pids[p11] = (int)i;
            }
        }
        uint32_t big = __ballot_sync(0xffffffffu, tx1 >= tx0 && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const float bX = __shfl_sync(0xffffffffu, r.X, src), bY = __shfl_sync(0xffffffffu, r.Y, src);
            const float bR = __shfl_sync(0xffffffffu, r.R, src);
            const float bcode = __shfl_sync(0xffffffffu, code, src);
            const int bid = __shfl_sync(0xffffffffu, (int)i, src);
            const int bx0 = __shfl_sync(0xffffffffu, tx0, src), bx1 = __shfl_sync(0xffffffffu, tx1, src);
            const int by0 = __shfl_sync(0xffffffffu, ty0, src), by1 = __shfl_sync(0xffffffffu, ty1, src);
            const int bw = bx1 - bx0 + 1, ncand = bw * (by1 - by0 + 1);
            const float4 rec = make_float4(bX, bY, bR, bcode);
            for (int k = lane; k < ncand; k += 32) {
                const int ty = by0 + k / bw, tx = bx0 + k % bw;
                if (tile_member(vp, bX, bY, bR, tx, ty)) {
                    const int t = ty * vp.ntx + tx;
                    const int pos = atomicAdd(&cur[t], 1);
                    lists[pos] = rec;
                    if (pids) pids[pos] = bid;
                }
            }
        }
    }
}

// Record code of a particle: species in the top 8 bits, normalised intensity in 24 bits.
__device__ __forceinline__ float record_code(int type, float itn) {
    uint32_t q = __float2uint_rn(__fmul_rn(itn, (float)kCodeMax));
    q = min(q, kCodeMax);
    return __uint_as_float(((uint32_t)type << 24) | q);
}

template <int S>
__global__ void __launch_bounds__(kThreads) k_scatter(SceneDev sc, FrameDev fr) {
    if (fr.status[kStatOverflow]) return;
    // cursor of this chunk's slice of every tile segment, relative to the start of the
    // view's segments (a view holds fewer than 2^31 pairs: the scan checks it)
    extern __shared__ int s_cur[];  // [g_n][n_tiles]
    __shared__ ViewParams s_view[kMaxGroup];
    __shared__ int64_t s_vbase[kMaxGroup];
    __shared__ int64_t s_tb[kMaxTypes + 1];
    const int b = blockIdx.x;
    const int v0 = blockIdx.y * fr.G;
    const int g_n = min(fr.G, fr.V - v0);
    const int nt = fr.n_tiles;
    for (int k = threadIdx.x; k < g_n * nt; k += blockDim.x) {
        const int g = k / nt, t = k - g * nt;
        const int64_t *seg = fr.offsets + (int64_t)(v0 + g) * nt;
        s_cur[k] = (int)(seg[t] - seg[0]) + fr.rel[((int64_t)(v0 + g) * fr.n_chunks + b) * nt + t];
    }
    if (threadIdx.x < g_n) {
        s_view[threadIdx.x] = fr.views[v0 + threadIdx.x];
        s_vbase[threadIdx.x] = fr.offsets[(int64_t)(v0 + threadIdx.x) * nt];
    }
    for (int k = threadIdx.x; k <= sc.n_types; k += blockDim.x) s_tb[k] = sc.type_begin[k];
    __syncthreads();

    const int64_t s = (int64_t)b * fr.chunk;
    const int64_t e = min(sc.n, s + fr.chunk);
    // two particles per thread per iteration in separate registers (see k_count)
    const int lane = threadIdx.x & 31;
    const int64_t stride = blockDim.x;
    int type = 0;
    int64_t i = s + threadIdx.x;
    float ax = 0.0f, ay = 0.0f, az = 0.0f, ah = 0.0f, ai = 0.0f;
    float bx = 0.0f, by = 0.0f, bz = 0.0f, bh = 0.0f, bi = 0.0f;
    if (i < e)
        ax = load1<S>(sc.x, i), ay = load1<S>(sc.y, i), az = load1<S>(sc.z, i), ah = load1<S>(sc.h, i),
        ai = load1<S>(sc.it, i);
    if (i + stride < e)
        bx = load1<S>(sc.x, i + stride), by = load1<S>(sc.y, i + stride), bz = load1<S>(sc.z, i + stride),
        bh = load1<S>(sc.h, i + stride), bi = load1<S>(sc.it, i + stride);
    for (; i - lane < e; i += 2 * stride) {
        if (i < e)
            while (type + 1 < sc.n_types && i >= s_tb[type + 1]) ++type;
        scatter_particle(i < e, i, ax, ay, az, ah, sc.emit ? __uint_as_float((uint32_t)i) : record_code(type, ai),
                         s_view, s_vbase, g_n, s_cur, nt, fr, lane);
        const int64_t ia = i + 2 * stride;
        if (ia < e)
            ax = load1<S>(sc.x, ia), ay = load1<S>(sc.y, ia), az = load1<S>(sc.z, ia), ah = load1<S>(sc.h, ia),
            ai = load1<S>(sc.it, ia);
        const int64_t j = i + stride;
        if (j - lane >= e) break;
        if (j < e)
            while (type + 1 < sc.n_types && j >= s_tb[type + 1]) ++type;
        scatter_particle(j < e, j, bx, by, bz, bh, sc.emit ? __uint_as_float((uint32_t)j) : record_code(type, bi),
                         s_view, s_vbase, g_n, s_cur, nt, fr, lane);
        const int64_t ib = i + 3 * stride;
        if (ib < e)
            bx = load1<S>(sc.x, ib), by = load1<S>(sc.y, ib), bz = load1<S>(sc.z, ib), bh = load1<S>(sc.h, ib),
            bi = load1<S>(sc.it, ib);
    }
}

template <int S> static cudaError_t scatter_impl(const SceneDev &sc, const FrameDev &fr, cudaStream_t st) {
    const size_t smem = (size_t)fr.G * fr.n_tiles * sizeof(int);
    cudaError_t err =
        ensure_smem_limit((const void *)k_scatter<S>, kBinSmemMax);
    if (err != cudaSuccess) return err;
    dim3 grid(fr.n_chunks, (fr.V + fr.G - 1) / fr.G);
    k_scatter<S><<<grid, kThreads, smem, st>>>(sc, fr);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------
// k_scatter_stable: the same slices, each in ascending particle index (as the per-thread
// index vectors of Section 3.2.1 are filled by walking each thread's particle range in
// order).  A CTA takes its chunk in rounds of kThreads consecutive particles (thread k
// holds particle round + k).  Per round and view
//   1. every thread rasterises its particle and counts its member tiles (a particle with
//      more than 2 x 2 candidate tiles is counted by its whole warp, one candidate per
//      lane);
//   2. a block scan of the counts places every pair in the round's pair list, which is
//      therefore in particle order; the pairs are staged in shared memory as (tile,
//      particle slot), kStableStage at a time;
//   3. every 32-pair slice finds, for each pair, the other pairs of its tile (the key
//      bits compared with ballots) and its rank among them; then one warp walks the
//      slices in order and, per tile of each slice, takes that many consecutive slots
//      from the tile's cursor;
//   4. all threads store the staged records at their slots (slice base + rank).
// With the chunk bases in chunk order, every tile list is in ascending particle index
// whatever the order in which CTAs and warps run, so images do not depend on it.  The
// ranking costs about twice the scatter's time; renders ask for it with SPLOTCH_STABLE.

constexpr int kStableStage = 2048;  // staged pairs per window
// shared memory beyond the cursors: round records, staged keys, slots and slice ranks
constexpr size_t kStableExtra = sizeof(float4) * kThreads + (sizeof(int) + 2 * sizeof(unsigned short)) * kStableStage;
// key bits compared per slice: tile indices are below kMaxTiles = 2^14, and bit 14 marks
// the lanes past the window's end
constexpr int kTileKeyBits = 15;
constexpr uint32_t kNoTile = 1u << 14;
static_assert(kMaxTiles <= (int)kNoTile, "tile keys need more bits");

// Member tiles of a particle whose candidate box is large, tested by the whole warp (one
// candidate per lane, candidates in row-major order).  With kStage false, returns the
// member count; with kStage true, stages the members of the window [w0, w0 + m) at pair
// indices off, off + 1, ... (off: the particle's first pair).
template <bool kStage>
__device__ __forceinline__ int big_members(const ViewParams &vp, float X, float Y, float R, int bx0, int bx1,
                                           int by0, int by1, int off, int w0, int m, int slot, int *s_key,
                                           unsigned short *s_slot, int lane) {
    const int bw = bx1 - bx0 + 1, bh = by1 - by0 + 1;
    const uint32_t lt = (1u << lane) - 1u;
    int run = off - w0;
    for (int dy = 0; dy < bh; ++dy) {
        for (int dx0 = 0; dx0 < bw; dx0 += 32) {
            const int tx = bx0 + dx0 + lane, ty = by0 + dy;
            const bool mem = dx0 + lane < bw && tile_member(vp, X, Y, R, tx, ty);
            const uint32_t bal = __ballot_sync(0xffffffffu, mem);
            if (kStage) {
                const int j = run + __popc(bal & lt);
                if (mem && (unsigned)j < (unsigned)m) {
                    s_key[j] = ty * vp.ntx + tx;
                    s_slot[j] = (unsigned short)slot;
                }
            }
            run += __popc(bal);
        }
    }
    return run - (off - w0);
}

template <int S>
__global__ void __launch_bounds__(kThreads) k_scatter_stable(SceneDev sc, FrameDev fr) {
    if (fr.status[kStatOverflow]) return;
    extern __shared__ __align__(16) unsigned char s_raw[];
    float4 *s_rec = reinterpret_cast<float4 *>(s_raw);                           // [kThreads]
    int *s_key = reinterpret_cast<int *>(s_rec + kThreads);                      // [kStableStage]
    unsigned short *s_slot = reinterpret_cast<unsigned short *>(s_key + kStableStage);  // [kStableStage]
    // per staged pair: its slice's leader lane for its tile (5 bits), its rank among the
    // slice's pairs of that tile (5 bits) and, at the leader, their count (6 bits)
    unsigned short *s_info = s_slot + kStableStage;                              // [kStableStage]
    // cursor of this chunk's slice of every tile segment, relative to the start of the
    // view's segments (a view holds fewer than 2^31 pairs: the scan checks it)
    int *s_cur = reinterpret_cast<int *>(s_info + kStableStage);                // [g_n][n_tiles]
    __shared__ ViewParams s_view[kMaxGroup];
    __shared__ int64_t s_vbase[kMaxGroup];
    __shared__ int64_t s_tb[kMaxTypes + 1];
    __shared__ int s_scan[33];
    const int b = blockIdx.x;
    const int v0 = blockIdx.y * fr.G;
    const int g_n = min(fr.G, fr.V - v0);
    const int nt = fr.n_tiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int k = tid; k < g_n * nt; k += blockDim.x) {
        const int g = k / nt, t = k - g * nt;
        const int64_t *seg = fr.offsets + (int64_t)(v0 + g) * nt;
        s_cur[k] = (int)(seg[t] - seg[0]) + fr.rel[((int64_t)(v0 + g) * fr.n_chunks + b) * nt + t];
    }
    if (tid < g_n) {
        s_view[tid] = fr.views[v0 + tid];
        s_vbase[tid] = fr.offsets[(int64_t)(v0 + tid) * nt];
    }
    for (int k = tid; k <= sc.n_types; k += blockDim.x) s_tb[k] = sc.type_begin[k];
    __syncthreads();

    const int64_t s = (int64_t)b * fr.chunk;
    const int64_t e = min(sc.n, s + fr.chunk);
    int type = 0;
    int64_t i = s + tid;
    float cx = 0.0f, cy = 0.0f, cz = 0.0f, ch = 0.0f, ci = 0.0f;
    if (i < e)
        cx = load1<S>(sc.x, i), cy = load1<S>(sc.y, i), cz = load1<S>(sc.z, i), ch = load1<S>(sc.h, i),
        ci = load1<S>(sc.it, i);
    for (int64_t r0 = s; r0 < e; r0 += kThreads, i += kThreads) {
        const bool valid = i < e;
        // the next round's attributes load while this round is binned
        float nx = 0.0f, ny = 0.0f, nz = 0.0f, nh = 0.0f, ni = 0.0f;
        const int64_t in = i + kThreads;
        if (in < e)
            nx = load1<S>(sc.x, in), ny = load1<S>(sc.y, in), nz = load1<S>(sc.z, in), nh = load1<S>(sc.h, in),
            ni = load1<S>(sc.it, in);
        if (valid)
            while (type + 1 < sc.n_types && i >= s_tb[type + 1]) ++type;
        const float code = sc.emit ? __uint_as_float((uint32_t)i) : record_code(type, ci);
        for (int g = 0; g < g_n; ++g) {
            const ViewParams &vp = s_view[g];
            Raster r;
            r.X = r.Y = r.R = 0.0f;
            int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
            if (valid && raster_one(vp, cx, cy, cz, ch, r)) {
                tx0 = tile_of(vp, r.i0), tx1 = tile_of(vp, r.i1);
                ty0 = tile_of(vp, r.j0), ty1 = tile_of(vp, r.j1);
            }
            const bool small = tx1 >= tx0 && tx1 - tx0 <= 1 && ty1 - ty0 <= 1;
            // member bits of a small particle: (tx0, ty0), (tx1, ty0), (tx0, ty1), (tx1, ty1)
            uint32_t mask = 0;
            if (small) {
                mask = (tile_member(vp, r.X, r.Y, r.R, tx0, ty0) ? 1u : 0u) |
                       (tx1 > tx0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty0) ? 2u : 0u) |
                       (ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx0, ty1) ? 4u : 0u) |
                       (tx1 > tx0 && ty1 > ty0 && tile_member(vp, r.X, r.Y, r.R, tx1, ty1) ? 8u : 0u);
            }
            int cnt = __popc(mask);
            const uint32_t big = __ballot_sync(0xffffffffu, tx1 >= tx0 && !small);
            for (uint32_t bb = big; bb; bb &= bb - 1) {
                const int src = __ffs(bb) - 1;
                const int n = big_members<false>(
                    vp, __shfl_sync(0xffffffffu, r.X, src), __shfl_sync(0xffffffffu, r.Y, src),
                    __shfl_sync(0xffffffffu, r.R, src), __shfl_sync(0xffffffffu, tx0, src),
                    __shfl_sync(0xffffffffu, tx1, src), __shfl_sync(0xffffffffu, ty0, src),
                    __shfl_sync(0xffffffffu, ty1, src), 0, 0, 0, 0, nullptr, nullptr, lane);
                if (lane == src) cnt = n;
            }
            int M = 0;
            const int off = block_excl_scan<int>(cnt, s_scan, &M);
            s_rec[tid] = make_float4(r.X, r.Y, r.R, code);
            float4 *lists = fr.lists + s_vbase[g];
            int *pids = fr.pids ? fr.pids + s_vbase[g] : nullptr;
            int *cur = s_cur + g * nt;
            for (int w0 = 0; w0 < M; w0 += kStableStage) {
                const int m = min(kStableStage, M - w0);
                // ---- 2. stage this window's pairs, in particle order
                if (mask) {
                    const int t00 = ty0 * vp.ntx + tx0;
                    int j = off - w0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!((mask >> q) & 1u)) continue;
                        if ((unsigned)j < (unsigned)m) {
                            s_key[j] = t00 + (q & 1) + ((q >> 1) ? vp.ntx : 0);
                            s_slot[j] = (unsigned short)tid;
                        }
                        ++j;
                    }
                }
                for (uint32_t bb = big; bb; bb &= bb - 1) {
                    const int src = __ffs(bb) - 1;
                    big_members<true>(vp, __shfl_sync(0xffffffffu, r.X, src), __shfl_sync(0xffffffffu, r.Y, src),
                                      __shfl_sync(0xffffffffu, r.R, src), __shfl_sync(0xffffffffu, tx0, src),
                                      __shfl_sync(0xffffffffu, tx1, src), __shfl_sync(0xffffffffu, ty0, src),
                                      __shfl_sync(0xffffffffu, ty1, src), __shfl_sync(0xffffffffu, off, src), w0, m,
                                      warp * 32 + src, s_key, s_slot, lane);
                }
                __syncthreads();
                // ---- 3a. per 32-pair slice: the pairs of each tile and their ranks
                for (int j0 = warp * 32; j0 < m; j0 += kThreads) {
                    const int j = j0 + lane;
                    const uint32_t t = j < m ? (uint32_t)s_key[j] : kNoTile;
                    const uint32_t peers = warp_peers<kTileKeyBits>(t);
                    const int leader = __ffs(peers) - 1;
                    if (j < m)
                        s_info[j] = (unsigned short)(leader | (__popc(peers & lt) << 5) |
                                                     ((lane == leader ? __popc(peers) : 0) << 10));
                }
                __syncthreads();
                // ---- 3b. slice bases in order: one warp; each slice's leader of a tile
                // takes its pairs' slots from the cursor and leaves the first in s_key
                if (warp == 0) {
                    for (int j0 = 0; j0 < m; j0 += 32) {
                        const int j = j0 + lane;
                        if (j < m) {
                            const int c = (int)(s_info[j] >> 10);
                            if (c) {
                                const int t = s_key[j];
                                const int base = cur[t];
                                cur[t] = base + c;
                                s_key[j] = base;
                            }
                        }
                    }
                }
                __syncthreads();
                // ---- 4. records to their slots: the leader's base plus the rank
                for (int j = tid; j < m; j += kThreads) {
                    const uint32_t inf = s_info[j];
                    const int pos = s_key[(j & ~31) + (int)(inf & 31u)] + (int)((inf >> 5) & 31u);
                    const int sl = s_slot[j];
                    lists[pos] = s_rec[sl];
                    if (pids) pids[pos] = (int)(r0 + sl);
                }
                __syncthreads();
            }
        }
        cx = nx, cy = ny, cz = nz, ch = nh, ci = ni;
    }
}

template <int S> static cudaError_t scatter_stable_impl(const SceneDev &sc, const FrameDev &fr, cudaStream_t st) {
    const size_t smem = (size_t)fr.G * fr.n_tiles * sizeof(int) + kStableExtra;
    cudaError_t err = ensure_smem_limit((const void *)k_scatter_stable<S>, kBinSmemMax + kStableExtra);
    if (err != cudaSuccess) return err;
    dim3 grid(fr.n_chunks, (fr.V + fr.G - 1) / fr.G);
    k_scatter_stable<S><<<grid, kThreads, smem, st>>>(sc, fr);
    return cudaGetLastError();
}

cudaError_t launch_scatter(int storage, const SceneDev &sc, const FrameDev &fr, bool stable, cudaStream_t st) {
    if (stable) {
        if (storage == 0) return scatter_stable_impl<0>(sc, fr, st);
        if (storage == 1) return scatter_stable_impl<1>(sc, fr, st);
        return scatter_stable_impl<2>(sc, fr, st);
    }
    if (storage == 0) return scatter_impl<0>(sc, fr, st);
    if (storage == 1) return scatter_impl<1>(sc, fr, st);
    return scatter_impl<2>(sc, fr, st);
}

// Resident CTAs per SM of the binning kernels with a histogram of `smem` bytes (the
// smaller of count and scatter, so both run their chunks in whole waves).
template <int S> static int bin_occupancy(size_t smem) {
    int a = 0, b = 0;
    if (ensure_smem_limit((const void *)k_count<S>, kBinSmemMax) != cudaSuccess ||
        ensure_smem_limit((const void *)k_scatter<S>, kBinSmemMax) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_count<S>, kThreads, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scatter<S>, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, std::min(a, b));
}

int bin_ctas_per_sm(int storage, size_t smem) {
    if (storage == 0) return bin_occupancy<0>(smem);
    if (storage == 1) return bin_occupancy<1>(smem);
    return bin_occupancy<2>(smem);
}

// ---------------------------------------------------------------------------------------
// Debug raster: X, Y, R, zc, colour (brightness x colormap of the stored normalised
// intensity), active, for one view.

template <int S>
__global__ void k_debug_raster(SceneDev sc, const ViewParams *__restrict__ view, float *out8) {
    const ViewParams vp = *view;
    constexpr int VEC = Store<S>::VEC;
    const int64_t n = sc.n;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * VEC; i < n;
         i += (int64_t)gridDim.x * blockDim.x * VEC) {
        float x[VEC], y[VEC], z[VEC], h[VEC], it[VEC];
        Store<S>::load(sc.x, i, x);
        Store<S>::load(sc.y, i, y);
        Store<S>::load(sc.z, i, z);
        Store<S>::load(sc.h, i, h);
        Store<S>::load(sc.it, i, it);
        for (int k = 0; k < VEC; ++k) {
            const int64_t p = i + k;
            if (p >= n) break;
            Raster r;
            r.X = r.Y = r.R = 0.0f;
            const bool act = raster_one(vp, x[k], y[k], z[k], h[k], r);
            int t = 0;
            while (t + 1 < sc.n_types && p >= sc.type_begin[t + 1]) ++t;
            const int len = sc.lut_len[t];
            const float f = it[k] * (float)(len - 1);
            const int kk = min((int)floorf(f), len - 2);
            const float tau = f - (float)kk;
            const float4 c0 = sc.lut[sc.lut_off[t] + kk], c1 = sc.lut[sc.lut_off[t] + kk + 1];
            out8[0 * n + p] = r.X;
            out8[1 * n + p] = r.Y;
            out8[2 * n + p] = r.R;
            out8[3 * n + p] = r.zc;
            out8[4 * n + p] = (1.0f - tau) * c0.x + tau * c1.x;
            out8[5 * n + p] = (1.0f - tau) * c0.y + tau * c1.y;
            out8[6 * n + p] = (1.0f - tau) * c0.z + tau * c1.z;
            out8[7 * n + p] = act ? 1.0f : 0.0f;
        }
    }
}

cudaError_t launch_debug_raster(int storage, const SceneDev &sc, const ViewParams *view, float *out8,
                                cudaStream_t st) {
    if (sc.n <= 0) return cudaSuccess;
    int64_t blocks = (sc.n + 255 * 8) / (256 * 8) + 1;
    if (blocks > 4096) blocks = 4096;
    if (storage == 0) k_debug_raster<0><<<(int)blocks, 256, 0, st>>>(sc, view, out8);
    else if (storage == 1) k_debug_raster<1><<<(int)blocks, 256, 0, st>>>(sc, view, out8);
    else k_debug_raster<2><<<(int)blocks, 256, 0, st>>>(sc, view, out8);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Depth-ordered binning (one view), for the transfer with absorption different from
// emission, where every tile list must run from the farthest particle to the nearest.
//   k_depth_records  per particle: record {X, Y, R, code}, depth key (all ones when the
//                    particle is not active) and its index;
//   (stable radix sort of the depth keys with the indices: equal depths keep index order)
//   k_sorted_counts  in that order: the gathered record and the number of tiles it belongs
//                    to (plus a zero past the end, so the exclusive scan ends with the total);
//   (exclusive scan of the counts: each particle's first output slot)
//   k_expand         each particle's records at its slots, keyed by tile id;
//   (stable radix sort by tile id: each tile's records stay in depth order)

// krange: {min, max} of the active particles' depth keys (atomicMin / atomicMax; the
// caller sets {all ones, 0} first), so that the sort covers only the bits they span.
template <int S>
__global__ void __launch_bounds__(256) k_depth_records(SceneDev sc, const ViewParams *__restrict__ views,
                                                       float4 *prec, uint32_t *dkey, uint32_t *pid,
                                                       uint32_t *krange) {
    __shared__ ViewParams s_v;
    __shared__ int64_t s_tb[kMaxTypes + 1];
    if (threadIdx.x == 0) s_v = views[0];
    for (int k = threadIdx.x; k <= sc.n_types; k += blockDim.x) s_tb[k] = sc.type_begin[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int type = 0;
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sc.n; i += stride) {
        while (type + 1 < sc.n_types && i >= s_tb[type + 1]) ++type;
        Raster r;
        const bool act = raster_one(s_v, load1<S>(sc.x, i), load1<S>(sc.y, i), load1<S>(sc.z, i),
                                    load1<S>(sc.h, i), r);
        prec[i] = make_float4(r.X, r.Y, r.R,
                              sc.emit ? __uint_as_float((uint32_t)i) : record_code(type, load1<S>(sc.it, i)));
        const uint32_t k = act ? depth_key(r.zc) : kInactiveKey;
        dkey[i] = k;
        pid[i] = (uint32_t)i;
        if (act) kmin = min(kmin, k), kmax = max(kmax, k);
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
        atomicMin(&krange[0], kmin);
        atomicMax(&krange[1], kmax);
    }
}

// Depth keys relative to the smallest active one (active: key - base in [0, span];
// inactive: span + 1, sorted last).
__global__ void k_rebase_keys(uint32_t *dkey, int64_t n, uint32_t base, uint32_t span) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = dkey[i];
        dkey[i] = k == kInactiveKey ? span + 1u : k - base;
    }
}

// Tiles of a rasterised particle, in row-major order over its tile box: the first
// `small` boxes (up to 2 x 2) by one lane, larger ones by the whole warp.
__device__ __forceinline__ void tile_box(const ViewParams &v, float X, float Y, float R, int &tx0, int &tx1,
                                         int &ty0, int &ty1) {
    int i0, i1, j0, j1;
    pixel_box(v, X, Y, R, i0, i1, j0, j1);
    tx0 = tile_of(v, i0), tx1 = tile_of(v, i1), ty0 = tile_of(v, j0), ty1 = tile_of(v, j1);
}

__global__ void __launch_bounds__(256) k_sorted_counts(const ViewParams *__restrict__ views,
                                                       const float4 *__restrict__ prec,
                                                       const uint32_t *__restrict__ skey,
                                                       const uint32_t *__restrict__ spid, int64_t n,
                                                       uint32_t inactive, float4 *srec, uint32_t *cnt) {
    __shared__ ViewParams s_v;
    if (threadIdx.x == 0) s_v = views[0];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[n] = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += wstride) {
        const int64_t q = base + lane;
        float4 rec = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (q < n && skey[q] != inactive) {
            rec = prec[spid[q]];
            tile_box(s_v, rec.x, rec.y, rec.z, tx0, tx1, ty0, ty1);
        }
        const bool small = tx1 >= tx0 && tx1 - tx0 <= 1 && ty1 - ty0 <= 1;
        uint32_t c = 0;
        if (small)
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) c += tile_member(s_v, rec.x, rec.y, rec.z, tx, ty) ? 1u : 0u;
        uint32_t big = __ballot_sync(0xffffffffu, tx1 >= tx0 && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const float bX = __shfl_sync(0xffffffffu, rec.x, src), bY = __shfl_sync(0xffffffffu, rec.y, src);
            const float bR = __shfl_sync(0xffffffffu, rec.z, src);
            const int bx0 = __shfl_sync(0xffffffffu, tx0, src), bx1 = __shfl_sync(0xffffffffu, tx1, src);
            const int by0 = __shfl_sync(0xffffffffu, ty0, src), by1 = __shfl_sync(0xffffffffu, ty1, src);
            const int bw = bx1 - bx0 + 1, ncand = bw * (by1 - by0 + 1);
            uint32_t mine = 0;
            for (int k = lane; k < ncand; k += 32)
                mine += tile_member(s_v, bX, bY, bR, bx0 + k % bw, by0 + k / bw) ? 1u : 0u;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, mine);
            if (lane == src) c = tot;
        }
        if (q < n) {
            srec[q] = rec;
            cnt[q] = c;
        }
    }
}

__global__ void __launch_bounds__(256) k_expand(const ViewParams *__restrict__ views,
                                                const float4 *__restrict__ srec, const uint32_t *__restrict__ poff,
                                                int64_t n, int64_t P, float4 *recs, uint32_t *tkey, uint32_t *tval,
                                                int *status) {
    __shared__ ViewParams s_v;
    if (threadIdx.x == 0) s_v = views[0];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += wstride) {
        const int64_t q = base + lane;
        float4 rec = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        uint32_t o0 = 0, c = 0;
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (q < n) {
            o0 = poff[q];
            c = poff[q + 1] - o0;
            if (c) {
                rec = srec[q];
                tile_box(s_v, rec.x, rec.y, rec.z, tx0, tx1, ty0, ty1);
            }
        }
        const bool small = c && tx1 >= tx0 && tx1 - tx0 <= 1 && ty1 - ty0 <= 1;
        if (small) {
            uint32_t k = 0;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    if (!tile_member(s_v, rec.x, rec.y, rec.z, tx, ty)) continue;
                    const uint32_t pos = o0 + k++;
                    if (k > c || (int64_t)pos >= P) {
                        atomicExch(&status[kStatOverflow], 1);
                        continue;
                    }
                    recs[pos] = rec;
                    tkey[pos] = (uint32_t)(ty * s_v.ntx + tx);
                    tval[pos] = pos;
                }
        }
        uint32_t big = __ballot_sync(0xffffffffu, c && tx1 >= tx0 && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const float4 b = make_float4(__shfl_sync(0xffffffffu, rec.x, src), __shfl_sync(0xffffffffu, rec.y, src),
                                         __shfl_sync(0xffffffffu, rec.z, src), __shfl_sync(0xffffffffu, rec.w, src));
            const uint32_t bo = __shfl_sync(0xffffffffu, o0, src), bc = __shfl_sync(0xffffffffu, c, src);
            const int bx0 = __shfl_sync(0xffffffffu, tx0, src), bx1 = __shfl_sync(0xffffffffu, tx1, src);
            const int by0 = __shfl_sync(0xffffffffu, ty0, src), by1 = __shfl_sync(0xffffffffu, ty1, src);
            const int bw = bx1 - bx0 + 1, ncand = bw * (by1 - by0 + 1);
            uint32_t k = 0;
            for (int kb = 0; kb < ncand; kb += 32) {
                const int kc = kb + lane;
                const int tx = bx0 + kc % bw, ty = by0 + kc / bw;
                const bool m = kc < ncand && tile_member(s_v, b.x, b.y, b.z, tx, ty);
                const uint32_t bal = __ballot_sync(0xffffffffu, m);
                if (m) {
                    const uint32_t kk = k + (uint32_t)__popc(bal & lt);
                    const uint32_t pos = bo + kk;
                    if (kk >= bc || (int64_t)pos >= P) {
                        atomicExch(&status[kStatOverflow], 1);
                    } else {
                        recs[pos] = b;
                        tkey[pos] = (uint32_t)(ty * s_v.ntx + tx);
                        tval[pos] = pos;
                    }
                }
                k += (uint32_t)__popc(bal);
            }
        }
    }
}

static int stream_grid(int64_t n, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * (2048 / threads)));
}

cudaError_t launch_depth_records(int storage, const SceneDev &sc, const ViewParams *views, float4 *prec,
                                 uint32_t *dkey, uint32_t *pid, uint32_t *krange, cudaStream_t st) {
    if (sc.n <= 0) return cudaSuccess;
    const int g = stream_grid(sc.n, 256);
    if (storage == 0) k_depth_records<0><<<g, 256, 0, st>>>(sc, views, prec, dkey, pid, krange);
    else if (storage == 1) k_depth_records<1><<<g, 256, 0, st>>>(sc, views, prec, dkey, pid, krange);
    else k_depth_records<2><<<g, 256, 0, st>>>(sc, views, prec, dkey, pid, krange);
    return cudaGetLastError();
}

cudaError_t launch_rebase_keys(uint32_t *dkey, int64_t n, uint32_t base, uint32_t span, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_rebase_keys<<<stream_grid(n, 256), 256, 0, st>>>(dkey, n, base, span);
    return cudaGetLastError();
}

cudaError_t launch_sorted_counts(const ViewParams *views, const float4 *prec, const uint32_t *skey,
                                 const uint32_t *spid, int64_t n, uint32_t inactive, float4 *srec, uint32_t *cnt,
                                 cudaStream_t st) {
    k_sorted_counts<<<stream_grid(std::max<int64_t>(1, n), 256), 256, 0, st>>>(views, prec, skey, spid, n, inactive,
                                                                               srec, cnt);
    return cudaGetLastError();
}

cudaError_t launch_expand(const ViewParams *views, const float4 *srec, const uint32_t *poff, int64_t n, int64_t P,
                          float4 *recs, uint32_t *tkey, uint32_t *tval, int *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_expand<<<stream_grid(n, 256), 256, 0, st>>>(views, srec, poff, n, P, recs, tkey, tval, status);
    return cudaGetLastError();
}

}  // namespace spl
