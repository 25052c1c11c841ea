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
// bulk copies (cp.async.bulk, double buffered, mbarrier completion with a bounded wait).
// Each stage is rendered in two phases:
//   A. small records (support < kBigR px): warps take 32 records at a time, enumerate
//      their (record, pixel row) pairs across lanes with a warp scan, and add e * w to
//      an FP32 tile accumulator in shared memory with atomic adds;
//   B. large records (support >= kBigR px, which carry most of the covered pixels):
//      each warp owns a band of 8 x 4 pixel blocks of the tile, one pixel per lane per
//      block, and gathers every large record over the blocks it overlaps into registers
//      (no atomics).
// The register sums join the shared accumulator at the end of the item.  The epilogue
// writes 1 - exp(-a) for the tile; slices of a split tile add their partial sums into a
// scratch tile and the last slice to finish writes the result.
#include "splotch_internal.cuh"

namespace spl {

constexpr float kBigR = 3.5f;

struct __align__(16) Slot {  // small record being enumerated by a warp
    float X, Y, R2, kr;
    float er, eg, eb, eps;
    int ilo, ihi, jlo, excl;
};

struct __align__(16) Big {  // large record queued for the register gather
    int ilo, ihi, jlo, jhi;
    float X, Y, R2, kr;
    float er, eg, eb, pad;
};

__device__ __forceinline__ int find_tile(const int *__restrict__ item_off, int N, int item) {
    int a = 0, b = N - 1;  // last gt with item_off[gt] <= item
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (__ldg(&item_off[m]) <= item) a = m; else b = m - 1;
    }
    return a;
}

__host__ __device__ __forceinline__ int acc_plane(int T) { return T * (T + 1) + 1; }

// 8 x 4 pixel blocks per warp for tile edge T (8 warps share ceil(T/8) * ceil(T/4) blocks)
__host__ __device__ __forceinline__ int blocks_per_warp(int T) {
    return (((T + 7) >> 3) * ((T + 3) >> 2) + kSplatWarps - 1) / kSplatWarps;
}

size_t splat_smem_bytes(int T) {
    return sizeof(float4) * 2 * kStage + sizeof(Slot) * kSplatWarps * 32 + sizeof(Big) * kStage +
           sizeof(short) * kSplatWarps * kStage + sizeof(float) * 3 * (size_t)acc_plane(T);
}

template <int NB>
__global__ void __launch_bounds__(kSplatThreads, 2) k_splat(SceneDev sc, FrameDev fr, int *queue, float *out,
                                                         int out_accum) {
    if (fr.status[kStatOverflow]) return;
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ uint64_t s_bar[2];
    __shared__ int s_item, s_last, s_nbig;
    __shared__ int s_next[2];
    __shared__ int s_wcnt[kSplatWarps];              // large records queued per warp band
    __shared__ int s_band[kSplatWarps][2];           // tile-local rows of each warp's blocks

    float4 *s_buf = reinterpret_cast<float4 *>(s_raw);                   // [2][kStage]
    Slot *s_slot = reinterpret_cast<Slot *>(s_buf + 2 * kStage);          // [warps][32]
    Big *s_big = reinterpret_cast<Big *>(s_slot + kSplatWarps * 32);      // [kStage]
    short *s_wlist = reinterpret_cast<short *>(s_big + kStage);           // [warps][kStage]
    float *s_acc = reinterpret_cast<float *>(s_wlist + kSplatWarps * kStage);  // [3][plane]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = fr.n_tiles;
    const int N = fr.V * nt;
    const int total_items = (int)fr.sizes[kSizeItems];
    const int64_t K = fr.sizes[kSizeK];
    const ViewParams g0 = fr.views[0];
    const int T = g0.T, W = g0.W, H = g0.H, ntx = g0.ntx;
    const int plane = acc_plane(T);
    const int stride = T + 1;

    // this warp's register blocks (tile-local origins), identical for every item
    const int bxn = (T + 7) >> 3, nbt = bxn * ((T + 3) >> 2);
    const int nbw = blocks_per_warp(T);
    const int lc = lane & 7, lr = lane >> 3;
    int bcol[NB], brow[NB];
    int band_lo = 1 << 30, band_hi = -(1 << 30);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int k = warp * nbw + b;
        const bool ok = b < nbw && k < nbt;
        bcol[b] = ok ? (k % bxn) * 8 : 1 << 28;
        brow[b] = ok ? (k / bxn) * 4 : 1 << 28;
        if (ok) {
            band_lo = min(band_lo, brow[b]);
            band_hi = max(band_hi, brow[b] + 3);
        }
    }

    if (lane == 0) {
        s_band[warp][0] = band_lo;
        s_band[warp][1] = band_hi;
        s_wcnt[warp] = 0;
    }
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
        s_nbig = 0;
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

        float ar[NB], ag[NB], ab[NB];
        unsigned pvalid = 0;  // bit b: this lane's pixel of block b lies in the tile and image
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            ar[b] = ag[b] = ab[b] = 0.0f;
            if (bcol[b] + lc < tw && brow[b] + lr < th) pvalid |= 1u << b;
        }

        for (int k = tid; k < 3 * plane; k += kSplatThreads) s_acc[k] = 0.0f;
        if (tid == 0) s_next[0] = s_next[1] = 0;
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
                s_next[nb] = 0;
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

            // ---- phase A: decode, queue large records, splat small ones -------------------
            const int ngroups = (cnt + 31) >> 5;
            for (;;) {
                int g = 0;
                if (lane == 0) g = atomicAdd(&s_next[cb], 1);
                g = __shfl_sync(0xffffffffu, g, 0);
                if (g >= ngroups) break;
                const int idx = g * 32 + lane;
                int nrows = 0;
                Slot me;
                if (idx < cnt) {
                    const float4 rec = recs[idx];
                    const float X = rec.x, Y = rec.y, R = rec.z;
                    const uint32_t code = __float_as_uint(rec.w);
                    // tight pixel range of the support inside the tile; eps exceeds the FP32
                    // rounding of X +- R at any position, so no covered pixel is left out
                    const float eps = 1e-3f + 2e-6f * (fabsf(X) + fabsf(Y) + R);
                    const int ilo = max(px0, (int)ceilf(clampf(X - R - 0.5f - eps, px0 - 1.0f, (float)(px0 + tw))));
                    const int ihi = min(px0 + tw - 1, (int)floorf(clampf(X + R - 0.5f + eps, px0 - 1.0f, (float)(px0 + tw))));
                    const int jlo = max(py0, (int)ceilf(clampf(Y - R - 0.5f - eps, py0 - 1.0f, (float)(py0 + th))));
                    const int jhi = min(py0 + th - 1, (int)floorf(clampf(Y + R - 0.5f + eps, py0 - 1.0f, (float)(py0 + th))));
                    const bool any = ilo <= ihi && jlo <= jhi;
                    const int type = (int)(code >> 24);
                    const float It = fminf((float)(code & kCodeMax) * (1.0f / (float)kCodeMax), 1.0f);
                    const int len = __ldg(&sc.lut_len[type]);
                    const float f = It * (float)(len - 1);
                    const int kk = min((int)f, len - 2);
                    const float tau = f - (float)kk;
                    const int lo = __ldg(&sc.lut_off[type]) + kk;
                    const float4 c0 = __ldg(&sc.lut[lo]);
                    const float4 c1 = __ldg(&sc.lut[lo + 1]);
                    const float R2 = __fmul_rn(R, R);
                    me.X = X; me.Y = Y; me.R2 = R2; me.kr = kexp / R2;
                    me.er = (1.0f - tau) * c0.x + tau * c1.x;
                    me.eg = (1.0f - tau) * c0.y + tau * c1.y;
                    me.eb = (1.0f - tau) * c0.z + tau * c1.z;
                    me.eps = eps;
                    me.ilo = ilo; me.ihi = ihi; me.jlo = jlo;
                    if (any && R >= kBigR) {
                        Big q;
                        q.ilo = ilo; q.ihi = ihi; q.jlo = jlo; q.jhi = jhi;
                        q.X = X; q.Y = Y; q.R2 = R2; q.kr = me.kr;
                        q.er = me.er; q.eg = me.eg; q.eb = me.eb; q.pad = 0.0f;
                        const int slotq = atomicAdd(&s_nbig, 1);
                        s_big[slotq] = q;
                        // queue it to every warp whose band of rows it meets
                        for (int w = 0; w < kSplatWarps; ++w) {
                            if (jhi < py0 + s_band[w][0] || jlo > py0 + s_band[w][1]) continue;
                            s_wlist[w * kStage + atomicAdd(&s_wcnt[w], 1)] = (short)slotq;
                        }
                    } else if (any) {
                        nrows = jhi - jlo + 1;
                    }
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
                    for (int st = 16; st; st >>= 1) {
                        const int cand = __shfl_sync(0xffffffffu, incl, l + st - 1);
                        if (cand <= itc) l += st;
                    }
                    if (it < total) {
                        const Slot P = sl[l];
                        const int row = P.jlo + (it - P.excl);
                        const float dy = __fsub_rn(__fadd_rn((float)row, 0.5f), P.Y);
                        const float dy2 = __fmul_rn(dy, dy);
                        // columns where dx^2 < R^2 - dy^2, widened by the rounding margin; the
                        // exact FP32 test below still decides every pixel
                        const float rem = fmaxf(P.R2 - dy2, 0.0f) + P.R2 * 4e-7f + 1e-12f;
                        const float half = rem * rsqrtf(rem + 1e-30f);
                        const float wide = half + P.eps;
                        const int a = max(P.ilo, (int)ceilf(clampf(P.X - 0.5f - wide, P.ilo - 1.0f, P.ihi + 1.0f)));
                        const int b = min(P.ihi, (int)floorf(clampf(P.X - 0.5f + wide, P.ilo - 1.0f, P.ihi + 1.0f)));
                        float *acc = s_acc + (row - py0) * stride - px0;
                        float fi = (float)a + 0.5f;
                        for (int i = a; i <= b; ++i, fi += 1.0f) {
                            const float dx = __fsub_rn(fi, P.X);
                            const float d2 = __fadd_rn(__fmul_rn(dx, dx), dy2);
                            if (d2 < P.R2) {
                                const float w = ex2_fast(d2 * P.kr);
                                atomicAdd(acc + i, P.er * w);
                                atomicAdd(acc + plane + i, P.eg * w);
                                atomicAdd(acc + 2 * plane + i, P.eb * w);
                            }
                        }
                    }
                }
                __syncwarp();
            }
            __syncthreads();

            // ---- phase B: register gather of the large records over this warp's blocks ------
            const int nmine = s_wcnt[warp];
            const short *mine = s_wlist + warp * kStage;
            for (int k = 0; k < nmine; ++k) {
                const Big *bq = &s_big[mine[k]];
                const int4 box = *reinterpret_cast<const int4 *>(&bq->ilo);
                const float4 pa = *reinterpret_cast<const float4 *>(&bq->X);
                const float4 pb = *reinterpret_cast<const float4 *>(&bq->er);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int c0 = px0 + bcol[b], r0 = py0 + brow[b];
                    if (c0 > box.y || c0 + 7 < box.x || r0 > box.w || r0 + 3 < box.z) continue;
                    const float dx = __fsub_rn((float)(c0 + lc) + 0.5f, pa.x);
                    const float dy = __fsub_rn((float)(r0 + lr) + 0.5f, pa.y);
                    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                    if (((pvalid >> b) & 1u) && d2 < pa.z) {
                        const float w = ex2_fast(d2 * pa.w);
                        ar[b] += pb.x * w;
                        ag[b] += pb.y * w;
                        ab[b] += pb.z * w;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) s_nbig = 0;
            if (lane == 0) s_wcnt[warp] = 0;
        }

        // register sums join the shared accumulator (each pixel has exactly one owner lane)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if ((pvalid >> b) & 1u) {
                const int o = (brow[b] + lr) * stride + bcol[b] + lc;
                s_acc[o] += ar[b];
                s_acc[plane + o] += ag[b];
                s_acc[2 * plane + o] += ab[b];
            }
        }
        __syncthreads();

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

typedef void (*SplatFn)(SceneDev, FrameDev, int *, float *, int);

static SplatFn splat_fn(int T) {
    const int nbw = blocks_per_warp(T);
    if (nbw <= 1) return k_splat<1>;
    if (nbw <= 2) return k_splat<2>;
    if (nbw <= 4) return k_splat<4>;
    if (nbw <= 8) return k_splat<8>;
    return k_splat<16>;
}

int splat_blocks_per_sm(int T) {
    const size_t smem = splat_smem_bytes(T);
    SplatFn fn = splat_fn(T);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kSplatThreads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_splat(const SceneDev &sc, const FrameDev &fr, int *queue, float *out, int out_accum,
                         int grid, cudaStream_t st) {
    const size_t smem = splat_smem_bytes(fr.T);
    SplatFn fn = splat_fn(fr.T);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    fn<<<grid, kSplatThreads, smem, st>>>(sc, fr, queue, out, out_accum);
    return cudaGetLastError();
}

__global__ void k_final(float *a, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = -expm1f(-a[i]);
}

cudaError_t launch_final(float *a, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_final<<<(int)blocks, 256, 0, st>>>(a, count);
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
