// Stable LSD radix sort of (64-bit key, 32-bit value) pairs on the device.
//
// The depth-ordered render (Section 2.1: with absorption different from emission the
// transfer equation must be applied along each line of sight in order) needs every tile
// list in depth order.  Records carry the key (tile << 32) | depth key; sorting the depth
// bits and then the tile bits, each pass stable, gives tile-major, far-to-near order (a
// first sort by particle index makes equal depths keep index order).
//
// One pass over 8 key bits:
//   k_digit_hist   each CTA counts the digits of its 4096 elements (warp-aggregated
//                  shared counters: the lanes of equal digit found with ballots), written
//                  digit-major: hist[digit * n_blocks + block];
//   k_scan_*       exclusive scan of hist, so hist[d * n_blocks + b] is where block b's
//                  elements of digit d start in the output;
//   k_digit_scatter each CTA re-reads its elements and writes them to their slots: an
//                  element's rank among equal digits follows input order (warps own
//                  consecutive ranges, lanes rank in order), so every pass is stable.
#include "splotch_internal.cuh"

namespace spl {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = 512;                       // consecutive elements per warp
constexpr int kSortTile = kSortWarps * kSortPerWarp;    // elements per CTA
constexpr int kSortRounds = kSortPerWarp / 32;
constexpr int kScanChunk = 4096;                        // entries per CTA in the scan

template <typename K> __device__ __forceinline__ uint32_t digit_of(K k, int shift) {
    return (uint32_t)(k >> shift) & 255u;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                            int n_blocks, uint32_t *hist) {
    __shared__ uint32_t s_cnt[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) s_cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kSortPerWarp;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? digit_of(keys[i], shift) : 256u;
        const uint32_t peers = warp_peers<9>(d);  // digits 0..255, 256 past the end
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSortThreads) hist[(int64_t)d * n_blocks + blockIdx.x] = s_cnt[d];
}

// Exclusive scan, three phases: per-chunk scans with chunk totals, a scan of the totals
// (one CTA), then the totals added back.
__device__ __forceinline__ uint32_t warp_scan_incl_u(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread over a 1024-thread CTA; *total gets the sum.
__device__ uint32_t block_scan_excl_u(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t incl = warp_scan_incl_u(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        const uint32_t wi = warp_scan_incl_u(w);
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t res = s_warp[warp] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(uint32_t *a, int64_t n, uint32_t *sums) {
    __shared__ uint32_t s_warp[33];
    const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
    uint32_t v[kScanChunk / 1024];
    uint32_t local = 0;
#pragma unroll
    for (int q = 0; q < kScanChunk / 1024; ++q) {
        const int64_t i = c0 + (int64_t)threadIdx.x * (kScanChunk / 1024) + q;
        v[q] = i < n ? a[i] : 0u;
        local += v[q];
    }
    uint32_t total;
    uint32_t run = block_scan_excl_u(local, s_warp, &total);
#pragma unroll
    for (int q = 0; q < kScanChunk / 1024; ++q) {
        const int64_t i = c0 + (int64_t)threadIdx.x * (kScanChunk / 1024) + q;
        if (i < n) a[i] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *sums, int m) {
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (int b = 0; b < m; b += 1024) {
        const int i = b + threadIdx.x;
        const uint32_t v = i < m ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_scan_excl_u(v, s_warp, &total);
        if (i < m) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void k_scan_add(uint32_t *a, int64_t n, const uint32_t *__restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * kScanChunk + threadIdx.x;
    const uint32_t s = sums[blockIdx.x];
    for (int64_t k = i; k < min(n, (int64_t)(blockIdx.x + 1) * kScanChunk); k += blockDim.x) a[k] += s;
}

// kGather: the last pass of a sort whose values index a payload: instead of the keys and
// values, write payload[value] to each element's slot (payload_out).
template <typename K, bool kGather>
__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const K *__restrict__ keys,
                                                               const uint32_t *__restrict__ vals, int64_t n,
                                                               int shift, int n_blocks,
                                                               const uint32_t *__restrict__ offs,
                                                               K *keys_out, uint32_t *vals_out,
                                                               const float4 *__restrict__ payload,
                                                               float4 *payload_out) {
    __shared__ uint32_t s_wc[kSortWarps][256];  // per warp: running count, then warp base
    __shared__ uint32_t s_off[256];             // output start of this CTA's digit d
    __shared__ uint32_t s_loc[256];             // start of digit d in the CTA's staged tile
    __shared__ uint32_t s_scan[33];
    __shared__ __align__(16) K s_key[kSortTile];  // staged keys, then staged values
    __shared__ uint8_t s_dig[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kSortWarps * 256; k += kSortThreads) (&s_wc[0][0])[k] = 0;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) s_off[d] = offs[(int64_t)d * n_blocks + blockIdx.x];
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int cnt = (int)min((int64_t)kSortTile, n - tile0);
    const int64_t base = tile0 + (int64_t)warp * kSortPerWarp;
    K k_r[kSortRounds];
    uint32_t v_r[kSortRounds], rank[kSortRounds];
    const uint32_t lt = (1u << lane) - 1u;
    // rank of each element among the equal digits of its warp's range, in input order
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        k_r[r] = ok ? keys[i] : (K)0;
        v_r[r] = ok ? vals[i] : 0u;
        const uint32_t d = ok ? digit_of(k_r[r], shift) : 256u;
        const uint32_t peers = warp_peers<9>(d);  // digits 0..255, 256 past the end
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (ok && lane == leader) {
            before = s_wc[warp][d];
            s_wc[warp][d] = before + (uint32_t)__popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[r] = before + (uint32_t)__popc(peers & lt);
        __syncwarp();  // this round's counter updates before the next round reads them
    }
    __syncthreads();
    // warp bases (elements of earlier warps with the same digit come first), the CTA's
    // digit totals, and their exclusive scan: where each digit starts in the staged tile
    {
        const int d = threadIdx.x;  // kSortThreads == 256 digits
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_wc[w][d];
            s_wc[w][d] = run;
            run += c;
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_scan[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t wv = lane < kSortWarps ? s_scan[lane] : 0u;
            uint32_t wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            if (lane < kSortWarps) s_scan[lane] = wi - wv;
        }
        __syncthreads();
        s_loc[d] = s_scan[warp] + incl - run;
    }
    __syncthreads();
    // stage the keys in digit order, then write each digit's run to consecutive slots
    uint32_t loc[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i >= n) continue;
        const uint32_t d = digit_of(k_r[r], shift);
        loc[r] = s_loc[d] + s_wc[warp][d] + rank[r];
        s_key[loc[r]] = k_r[r];
        s_dig[loc[r]] = (uint8_t)d;
    }
    __syncthreads();
    if (!kGather) {
        for (int l = threadIdx.x; l < cnt; l += kSortThreads) {
            const uint32_t d = s_dig[l];
            keys_out[s_off[d] + (uint32_t)l - s_loc[d]] = s_key[l];
        }
    }
    __syncthreads();
    uint32_t *s_val = reinterpret_cast<uint32_t *>(s_key);
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) s_val[loc[r]] = v_r[r];
    }
    __syncthreads();
    for (int l = threadIdx.x; l < cnt; l += kSortThreads) {
        const uint32_t d = s_dig[l];
        const uint32_t g = s_off[d] + (uint32_t)l - s_loc[d];
        if (kGather)
            payload_out[g] = payload[s_val[l]];
        else
            vals_out[g] = s_val[l];
    }
}

static int sort_blocks(int64_t n) { return (int)((n + kSortTile - 1) / kSortTile); }

size_t sort_temp_bytes(int64_t n) {
    const int64_t h = (int64_t)256 * std::max(1, sort_blocks(n));
    const int64_t chunks = (h + kScanChunk - 1) / kScanChunk;
    return sizeof(uint32_t) * (size_t)(h + chunks) + 256;
}

// Sorts keys[0, n) with their values by key bits [bit_lo, bit_hi), stably, ping-ponging
// with the alternate buffers; *in_alt tells which pair of buffers holds the result.
template <typename K>
static cudaError_t sort_impl(K *keys, K *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int bit_lo,
                             int bit_hi, void *temp, cudaStream_t st, bool *in_alt,
                             const float4 *payload = nullptr, float4 *payload_out = nullptr) {
    *in_alt = false;
    if (n <= 1 || bit_lo >= bit_hi) {
        if (payload && n > 0) return launch_gather_records(payload, vals, n, payload_out, st);
        return cudaSuccess;
    }
    const int nb = sort_blocks(n);
    const int64_t h = (int64_t)256 * nb;
    const int chunks = (int)((h + kScanChunk - 1) / kScanChunk);
    uint32_t *hist = (uint32_t *)temp;
    uint32_t *sums = hist + h;
    K *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int shift = bit_lo; shift < bit_hi; shift += 8) {
        k_digit_hist<K><<<nb, kSortThreads, 0, st>>>(ka, n, shift, nb, hist);
        k_scan_chunks<<<chunks, 1024, 0, st>>>(hist, h, sums);
        k_scan_sums<<<1, 1024, 0, st>>>(sums, chunks);
        k_scan_add<<<chunks, 1024, 0, st>>>(hist, h, sums);
        if (payload && shift + 8 >= bit_hi)
            k_digit_scatter<K, true><<<nb, kSortThreads, 0, st>>>(ka, va, n, shift, nb, hist, kb, vb, payload,
                                                                 payload_out);
        else
            k_digit_scatter<K, false><<<nb, kSortThreads, 0, st>>>(ka, va, n, shift, nb, hist, kb, vb, nullptr,
                                                                  nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::swap(ka, kb);
        std::swap(va, vb);
        *in_alt = !*in_alt;
    }
    return cudaSuccess;
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int bit_lo, int bit_hi, void *temp, cudaStream_t st, bool *in_alt) {
    return sort_impl<uint64_t>(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, temp, st, in_alt);
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int bit_lo, int bit_hi, void *temp, cudaStream_t st, bool *in_alt) {
    return sort_impl<uint32_t>(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, temp, st, in_alt);
}

cudaError_t radix_sort_gather(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                              int bit_lo, int bit_hi, void *temp, const float4 *payload, float4 *payload_out,
                              cudaStream_t st) {
    bool alt = false;
    return sort_impl<uint32_t>(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, temp, st, &alt, payload,
                               payload_out);
}

size_t scan_temp_bytes(int64_t n) {
    return sizeof(uint32_t) * (size_t)((std::max<int64_t>(1, n) + kScanChunk - 1) / kScanChunk) + 256;
}

// In-place exclusive scan of a[0, n) (the total must stay below 2^32).
cudaError_t exclusive_scan_u32(uint32_t *a, int64_t n, void *temp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int chunks = (int)((n + kScanChunk - 1) / kScanChunk);
    uint32_t *sums = (uint32_t *)temp;
    k_scan_chunks<<<chunks, 1024, 0, st>>>(a, n, sums);
    k_scan_sums<<<1, 1024, 0, st>>>(sums, chunks);
    k_scan_add<<<chunks, 1024, 0, st>>>(a, n, sums);
    return cudaGetLastError();
}

}  // namespace spl
