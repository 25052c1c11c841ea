// Per-tile Gaussian splat and final transform for the Splotch hot path.
//
// Section 3.1: each tile's particle list is rendered by one worker that owns the
// tile's pixels, so pixel updates never race with another tile.  Section 3.2.2: a
// draw adds particle colour x scalar weight to the pixel.  Section 2.1: the weight is
// a Gaussian of the distance to the particle centre over the radius-dependent area.
//
// GB300 layout: one persistent CTA per SM slot pulls work items from a queue.  A work
// item is a tile, or a K-record slice of a crowded tile (so dense clusters do not
// serialise on one CTA).  The item's records are staged from HBM into shared memory by
// bulk copies (cp.async.bulk, double buffered, mbarrier completion with a bounded
// wait); each warp takes 32 records, enumerates their (record, pixel row) pairs across
// lanes with a warp scan and adds e * w to an FP32 tile accumulator in shared memory.
// The epilogue writes 1 - exp(-a) for the tile; slices of a split tile add their
// partial sums into a scratch tile and the last slice to finish writes the result.
#include "splotch_internal.cuh"

namespace spl {

struct __align__(16) Slot {
    float X, Y, R2, kr;
    float er, eg, eb;
    int ci0;
    int ci1, cj0, excl, pad;
};

__device__ __forceinline__ int find_tile(const int *__restrict__ item_off, int N, int item) {
    int a = 0, b = N - 1;  // last gt with item_off[gt] <= item
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (__ldg(&item_off[m]) <= item) a = m; else b = m - 1;
    }
    return a;
}

__device__ __forceinline__ int acc_plane(int T) { return T * (T + 1) + 1; }

size_t splat_smem_bytes(int T) {
    return sizeof(float4) * 2 * kStage + sizeof(Slot) * kSplatWarps * 32 +
           sizeof(float) * 3 * (size_t)(T * (T + 1) + 1);
}

__global__ void __launch_bounds__(kSplatThreads) k_splat(SceneDev sc, FrameDev fr, int *queue, float *out,
                                                         int out_accum) {
    if (fr.status[kStatOverflow]) return;
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ uint64_t s_bar[2];
    __shared__ int s_item, s_last;

    float4 *s_buf = reinterpret_cast<float4 *>(s_raw);                    // [2][kStage]
    Slot *s_slot = reinterpret_cast<Slot *>(s_buf + 2 * kStage);           // [warps][32]
    float *s_acc = reinterpret_cast<float *>(s_slot + kSplatWarps * 32);   // [3][plane]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = fr.n_tiles;
    const int N = fr.V * nt;
    const int total_items = (int)fr.sizes[kSizeItems];
    const int64_t K = fr.sizes[kSizeK];
    const ViewParams g0 = fr.views[0];
    const int T = g0.T, W = g0.W, H = g0.H, ntx = g0.ntx;
    const int plane = acc_plane(T);
    const int stride = T + 1;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t phase0 = 0, phase1 = 0;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;

        const int gt = find_tile(fr.item_off, N, item);
        const int v = gt / nt, t = gt - v * nt;
        const int chunk = item - fr.item_off[gt];
        const int n_it = fr.item_off[gt + 1] - fr.item_off[gt];
        const int slot = fr.split_slot[gt];
        const float kexp = fr.views[v].kexp;
        const int tx = t % ntx, ty = t / ntx;
        const int px0 = tx * T, py0 = ty * T;
        const int tw = min(T, W - px0), th = min(T, H - py0);
        const int64_t seg1 = fr.offsets[gt + 1];
        const int64_t e0 = fr.offsets[gt] + (int64_t)chunk * K;
        const int nrec = (int)(min(seg1, e0 + K) - e0);
        const int nst = (nrec + kStage - 1) / kStage;

        for (int k = tid; k < 3 * plane; k += kSplatThreads) s_acc[k] = 0.0f;
        if (tid == 0 && nrec > 0) {
            const int c0 = min(kStage, nrec);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[0], (uint32_t)c0 * 16u);
            bulk_g2s(s_buf, fr.lists + e0, (uint32_t)c0 * 16u, &s_bar[0]);
        }
        __syncthreads();

        for (int si = 0; si < nst; ++si) {
            const int cb = si & 1;
            if (tid == 0 && si + 1 < nst) {
                const int nb = (si + 1) & 1;
                const int cn = min(kStage, nrec - (si + 1) * kStage);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&s_bar[nb], (uint32_t)cn * 16u);
                bulk_g2s(s_buf + nb * kStage, fr.lists + e0 + (int64_t)(si + 1) * kStage,
                         (uint32_t)cn * 16u, &s_bar[nb]);
            }
            const bool ok = mbar_wait_bounded(&s_bar[cb], cb ? phase1 : phase0, kWaitCycles);
            if (cb) phase1 ^= 1u; else phase0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(&fr.status[kStatTimeout], 1);
                return;
            }
            const int cnt = min(kStage, nrec - si * kStage);
            const float4 *recs = s_buf + cb * kStage;
            Slot *sl = s_slot + warp * 32;
            for (int g = warp; g * 32 < cnt; g += kSplatWarps) {
                const int idx = g * 32 + lane;
                int nrows = 0;
                Slot me;
                if (idx < cnt) {
                    const float4 rec = recs[idx];
                    const float X = rec.x, Y = rec.y, R = rec.z;
                    const uint32_t code = __float_as_uint(rec.w);
                    int i0, i1, j0, j1;
                    pixel_box(g0, X, Y, R, i0, i1, j0, j1);
                    const int ci0 = max(i0, px0), ci1 = min(i1, px0 + tw - 1);
                    const int cj0 = max(j0, py0), cj1 = min(j1, py0 + th - 1);
                    if (ci0 <= ci1 && cj0 <= cj1) nrows = cj1 - cj0 + 1;
                    const int type = (int)(code >> 24);
                    const float It = fminf((float)(code & kCodeMax) * (1.0f / (float)kCodeMax), 1.0f);
                    const int len = __ldg(&sc.lut_len[type]);
                    const float f = It * (float)(len - 1);
                    const int kk = min((int)f, len - 2);
                    const float tau = f - (float)kk;
                    const float4 c0 = __ldg(&sc.lut[__ldg(&sc.lut_off[type]) + kk]);
                    const float4 c1 = __ldg(&sc.lut[__ldg(&sc.lut_off[type]) + kk + 1]);
                    const float R2 = __fmul_rn(R, R);
                    me.X = X; me.Y = Y; me.R2 = R2; me.kr = kexp / R2;
                    me.er = (1.0f - tau) * c0.x + tau * c1.x;
                    me.eg = (1.0f - tau) * c0.y + tau * c1.y;
                    me.eb = (1.0f - tau) * c0.z + tau * c1.z;
                    me.ci0 = ci0; me.ci1 = ci1; me.cj0 = cj0;
                }
                const int incl = warp_incl_scan_i(nrows);
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                if (total == 0) continue;
                if (nrows) {
                    me.excl = incl - nrows;
                    sl[lane] = me;
                }
                __syncwarp();
                for (int base = 0; base < total; base += 32) {
                    const int it = base + lane;
                    const int itc = min(it, total - 1);
                    int l = 0;
#pragma unroll
                    for (int s = 16; s; s >>= 1) {
                        const int cand = __shfl_sync(0xffffffffu, incl, l + s - 1);
                        if (cand <= itc) l += s;
                    }
                    if (it < total) {
                        const Slot P = sl[l];
                        const int row = P.cj0 + (it - P.excl);
                        const float dy = __fsub_rn(__fadd_rn((float)row, 0.5f), P.Y);
                        const float dy2 = __fmul_rn(dy, dy);
                        float *a = s_acc + (row - py0) * stride - px0;
                        for (int i = P.ci0; i <= P.ci1; ++i) {
                            const float dx = __fsub_rn(__fadd_rn((float)i, 0.5f), P.X);
                            const float d2 = __fadd_rn(__fmul_rn(dx, dx), dy2);
                            if (d2 < P.R2) {
                                const float w = exp2f(d2 * P.kr);
                                atomicAdd(a + i, P.er * w);
                                atomicAdd(a + plane + i, P.eg * w);
                                atomicAdd(a + 2 * plane + i, P.eb * w);
                            }
                        }
                    }
                }
                __syncwarp();
            }
            __syncthreads();
        }

        // epilogue: final transform of the tile, or merge of a split tile's slices
        float *o = out + (int64_t)v * H * W * 3;
        const int rowlen = 3 * tw;
        if (slot < 0) {
            for (int k = tid; k < th * rowlen; k += kSplatThreads) {
                const int r = k / rowlen, cc = k - r * rowlen;
                const int col = cc / 3, ch = cc - col * 3;
                const float a = s_acc[ch * plane + r * stride + col];
                o[((int64_t)(py0 + r) * W + px0) * 3 + cc] = out_accum ? a : -expm1f(-a);
            }
        } else {
            float *scr = fr.scratch + (int64_t)slot * 3 * T * T;
            for (int k = tid; k < 3 * T * T; k += kSplatThreads) {
                const int ch = k / (T * T), rem = k - ch * T * T;
                const int r = rem / T, col = rem - r * T;
                const float a = s_acc[ch * plane + r * stride + col];
                if (a != 0.0f) atomicAdd(&scr[k], a);
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = (atomicAdd(&fr.tickets[slot], 1) == n_it - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                for (int k = tid; k < th * rowlen; k += kSplatThreads) {
                    const int r = k / rowlen, cc = k - r * rowlen;
                    const int col = cc / 3, ch = cc - col * 3;
                    const float a = __ldcg(&scr[ch * T * T + r * T + col]);
                    o[((int64_t)(py0 + r) * W + px0) * 3 + cc] = out_accum ? a : -expm1f(-a);
                }
                __syncthreads();
                for (int k = tid; k < 3 * T * T; k += kSplatThreads) scr[k] = 0.0f;
                if (tid == 0) fr.tickets[slot] = 0;
            }
        }
        __syncthreads();
    }
}

int splat_blocks_per_sm(int T) {
    const size_t smem = splat_smem_bytes(T);
    if (cudaFuncSetAttribute(k_splat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_splat, kSplatThreads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_splat(const SceneDev &sc, const FrameDev &fr, int *queue, float *out, int out_accum,
                         int grid, cudaStream_t st) {
    const size_t smem = splat_smem_bytes(fr.T);
    cudaError_t err = cudaFuncSetAttribute(k_splat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_splat<<<grid, kSplatThreads, smem, st>>>(sc, fr, queue, out, out_accum);
    return cudaGetLastError();
}

// A CTA waits on an mbarrier that expects one arrival nobody makes: the bounded wait must
// give up and report, leaving the context usable.
__global__ void k_selftest_wait(long long limit, int *result) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit);
    if (threadIdx.x == 0) *result = ok ? 1 : 2;
}

cudaError_t launch_selftest_wait(long long limit, int *result, cudaStream_t st) {
    k_selftest_wait<<<1, 32, 0, st>>>(limit, result);
    return cudaGetLastError();
}

}  // namespace spl
