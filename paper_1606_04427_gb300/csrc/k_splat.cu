// Per-tile Gaussian splat and final transform for the Splotch hot path.
//
// Section 3.1: each tile's particle list is rendered by one worker that owns the
// tile's pixels, so pixel updates never race with another tile.  Section 3.2.2: a
// draw adds particle colour x scalar weight to the pixel.  Section 2.1: the weight is
// a Gaussian of the distance to the particle centre over the radius-dependent area.
//
// GB300 layout: persistent CTAs pull work items from a queue.  A work item is a tile,
// or a K-record slice of a crowded tile (so dense clusters do not serialise on one
// worker); slices of a split tile add their partial sums into a scratch tile and the
// last slice to finish writes the result.  Records are staged from HBM into shared
// memory by bulk copies (cp.async.bulk, double buffered, mbarrier completion with a
// bounded wait).  The paper's worker is a thread; here pixels are owned by lanes, each
// accumulating its pixels in registers (no atomics: a pixel has exactly one owner), in
// blocks of 8 x 4 pixels, one pixel of each block per lane.  Two kernels:
//   k_splat_warp  tiles up to 32 px: one warp owns a square of up to 16 x 16 pixels (a
//                 tile, or a quarter of a larger one) and runs its records grouped by
//                 the rectangle of blocks they cover (below);
//   k_splat       tiles above 32 px: the 8 warps of a CTA share a tile by block rows,
//                 each record queued to the warps whose rows it meets.
// In clustered data most pixels receive hundreds of contributions per frame, where a
// shared-memory scatter would serialise on atomic conflicts.
#include "splotch_internal.cuh"

namespace spl {

// ---------------------------------------------------------------------------------------
// CTA-per-item splat for tiles above 32 px.  Per stage of kStage records:
//   1. decode: one thread per record computes the record's pixel box inside the tile, its
//      colour (brightness x colormap, or the particle's emission) and Gaussian scale, and
//      appends the record to the list of every warp owning a block row the box meets
//      (block row r: warp r mod 8);
//   2. gather: each warp walks its list; for every block of its own that the box
//      overlaps, each lane tests its pixel with the FP32 coverage rule and adds e * w
//      to its registers.

struct __align__(16) Rec {
    int ilo, ihi, jlo, jhi;  // tile-local box
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

// blocks of 8 x 4 pixels; warp w owns block rows w, w + 8, ...: NR block rows of NC
// blocks each (NC = ceil(T / 8), NR = ceil(ceil(T / 4) / 8))
__host__ __device__ __forceinline__ int block_cols(int T) { return (T + 7) >> 3; }
__host__ __device__ __forceinline__ int block_rows_per_warp(int T) {
    return (((T + 3) >> 2) + kSplatWarps - 1) / kSplatWarps;
}

size_t splat_smem_bytes(int) {
    return sizeof(float4) * 2 * kStage + sizeof(Rec) * kStage + sizeof(short) * kSplatWarps * kStage;
}

// pixel centre coordinate that no support reaches (its square overflows to +inf)
constexpr float kFar = 1e30f;

// Output of a pixel's accumulation a: mode 0 writes 1 - exp(-a) (final transform),
// 1 writes a, 2 adds a to what the pixel holds (several renders summed in one image).
__device__ __forceinline__ void put_pixel(float *p, float a, int mode) {
    *p = mode == 2 ? *p + a : (mode ? a : -expm1f(-a));
}

template <int NR, int NC>
__global__ void __launch_bounds__(kSplatThreads, 3) k_splat(SceneDev sc, FrameDev fr, int *queue, float *out,
                                                         int out_accum) {
    if (fr.status[kStatOverflow] || fr.status[kStatTimeout]) return;  // no complete tile lists
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ uint64_t s_bar[2];
    __shared__ int s_item, s_last;

    float4 *s_buf = reinterpret_cast<float4 *>(s_raw);             // [2][kStage]
    Rec *s_rec = reinterpret_cast<Rec *>(s_buf + 2 * kStage);       // [kStage]
    short *s_wl = reinterpret_cast<short *>(s_rec + kStage);        // [warps][kStage]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = fr.n_tiles;
    const int N = fr.V * nt;
    const int total_items = (int)fr.sizes[kSizeItems];
    const int64_t K = fr.sizes[kSizeK];
    const ViewParams g0 = fr.views[0];
    const int T = g0.T, W = g0.W, H = g0.H, ntx = g0.ntx;
    const int lc = lane & 7, lr = lane >> 3;

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
        const int qi = s_item;
        if (qi >= total_items) break;
        const int item = fr.order ? __ldg(&fr.order[qi]) : qi;

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

        // this lane's pixels: column c * 8 + lc of block row warp + 8 rr (tile rows
        // 4 (warp + 8 rr) + lr); pixels outside the tile get a centre no support reaches
        float fx[NC], fy[NR], ar[NR][NC], ag[NR][NC], ab[NR][NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) fx[c] = c * 8 + lc < tw ? (float)(px0 + c * 8 + lc) + 0.5f : kFar;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            const int row = 4 * (warp + kSplatWarps * rr) + lr;
            fy[rr] = row < th ? (float)(py0 + row) + 0.5f : kFar;
#pragma unroll
            for (int c = 0; c < NC; ++c) ar[rr][c] = ag[rr][c] = ab[rr][c] = 0.0f;
        }

        if (tid == 0 && nrec > 0) {
            const int c0 = min(kStage, nrec);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[0], (uint32_t)c0 * 16u);
            bulk_g2s(s_buf, fr.lists + e0, (uint32_t)c0 * 16u, &s_bar[0]);
        }

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

            // ---- 1. decode; queue each record to the warps owning the block rows it meets
            for (int idx = tid; idx < cnt; idx += kSplatThreads) {
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
                if (ilo > ihi || jlo > jhi) {
                    s_rec[idx].jlo = 1;  // no pixel of the tile: no warp takes it
                    s_rec[idx].jhi = 0;
                    continue;
                }
                int type;
                float3 e;
                if (sc.emit) {
                    const float4 em = __ldg(&sc.emit[code]);  // the code is the particle index
                    type = __float_as_int(em.w);
                    e = make_float3(em.x, em.y, em.z);
                } else {
                    type = (int)(code >> 24);
                    const float It = fminf((float)(code & kCodeMax) * (1.0f / (float)kCodeMax), 1.0f);
                    const bool per_view = fr.vlut != nullptr;  // the view's colormap in a plan
                    const int vi = v * sc.n_types + type;
                    const float4 *lut = per_view ? fr.vlut : sc.lut;
                    const int len = per_view ? __ldg(&fr.vlut_len[vi]) : __ldg(&sc.lut_len[type]);
                    const int off = per_view ? __ldg(&fr.vlut_off[vi]) : __ldg(&sc.lut_off[type]);
                    const float f = It * (float)(len - 1);
                    const int kk = min((int)f, len - 2);
                    const float tau = f - (float)kk;
                    const float4 c0 = __ldg(&lut[off + kk]);
                    const float4 c1 = __ldg(&lut[off + kk + 1]);
                    e = make_float3((1.0f - tau) * c0.x + tau * c1.x, (1.0f - tau) * c0.y + tau * c1.y,
                                    (1.0f - tau) * c0.z + tau * c1.z);
                }
                Rec q;
                q.ilo = ilo - px0;
                q.ihi = ihi - px0;
                q.jlo = jlo - py0;
                q.jhi = jhi - py0;
                q.X = X;
                q.Y = Y;
                q.R2 = __fmul_rn(R, R);
                q.kr = __fdividef(kexp, q.R2);
                const float vs = fr.vscale ? __ldg(&fr.vscale[v * sc.n_types + type]) : 1.0f;
                q.er = e.x * vs;
                q.eg = e.y * vs;
                q.eb = e.z * vs;
                q.pad = 0.0f;
                s_rec[idx] = q;
            }
            __syncthreads();
            // this warp's list: the records whose box meets one of its block rows, in
            // record order (so every pixel sums its records in list order)
            int nmine = 0;
            short *mine = s_wl + warp * kStage;
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const int idx = j0 + lane;
                bool meets = false;
                if (idx < cnt) {
                    const int jl = s_rec[idx].jlo, jh = s_rec[idx].jhi;
                    if (jl <= jh) {
                        const int br0 = jl >> 2, nbr = (jh >> 2) - br0 + 1;
                        meets = nbr >= kSplatWarps || ((warp - br0) & (kSplatWarps - 1)) < nbr;
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, meets);
                if (meets) mine[nmine + __popc(bal & ((1u << lane) - 1u))] = (short)idx;
                nmine += __popc(bal);
            }
            __syncwarp();

            // ---- 2. gather: this warp's list over this warp's blocks ---------------------
            for (int k = 0; k < nmine; ++k) {
                const Rec *q = &s_rec[mine[k]];
                const int4 box = *reinterpret_cast<const int4 *>(&q->ilo);
                const float4 pa = *reinterpret_cast<const float4 *>(&q->X);
                const float4 pb = *reinterpret_cast<const float4 *>(&q->er);
                // block columns the box overlaps, as a bit mask (uniform over the warp)
                const uint32_t cm = (2u << (box.y >> 3)) - (1u << (box.x >> 3));
#pragma unroll
                for (int rr = 0; rr < NR; ++rr) {
                    const int r0 = 4 * (warp + kSplatWarps * rr);
                    if (NR > 1 && (r0 > box.w || r0 + 3 < box.z)) continue;
                    const float dy = __fsub_rn(fy[rr], pa.y);
                    const float dy2 = __fmul_rn(dy, dy);
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (!(cm & (1u << c))) continue;
                        const float dx = __fsub_rn(fx[c], pa.x);
                        const float d2 = __fadd_rn(__fmul_rn(dx, dx), dy2);
                        if (d2 < pa.z) {
                            const float w = ex2_fast(d2 * pa.w);
                            ar[rr][c] += pb.x * w;
                            ag[rr][c] += pb.y * w;
                            ab[rr][c] += pb.z * w;
                        }
                    }
                }
            }
            __syncthreads();
        }

        // epilogue: final transform of this lane's pixels, or merge of a split tile
        float *o = out + (int64_t)v * H * W * 3;
        if (slot < 0) {
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) {
                const int row = 4 * (warp + kSplatWarps * rr) + lr;
                if (row >= th) continue;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * 8 + lc >= tw) continue;
                    float *p = o + ((int64_t)(py0 + row) * W + px0 + c * 8 + lc) * 3;
                    put_pixel(p, ar[rr][c], out_accum);
                    put_pixel(p + 1, ag[rr][c], out_accum);
                    put_pixel(p + 2, ab[rr][c], out_accum);
                }
            }
        } else {
            unsigned long long *scr = fr.scratch + (int64_t)slot * 6 * T * T;
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) {
                const int row = 4 * (warp + kSplatWarps * rr) + lr;
                if (row >= th) continue;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c * 8 + lc >= tw) continue;
                    const int pix = row * T + c * 8 + lc;
                    fix_add(&scr[2 * pix], ar[rr][c]);
                    fix_add(&scr[2 * (T * T + pix)], ag[rr][c]);
                    fix_add(&scr[2 * (2 * T * T + pix)], ab[rr][c]);
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = (atomicAdd(&fr.tickets[slot], 1) == n_it - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                const int rowlen = 3 * tw;
                for (int k = tid; k < th * rowlen; k += kSplatThreads) {
                    const int r = k / rowlen, cc = k - r * rowlen;
                    const int col = cc / 3, ch = cc - col * 3;
                    const float a = fix_value(&scr[2 * (ch * T * T + r * T + col)]);
                    put_pixel(&o[((int64_t)(py0 + r) * W + px0) * 3 + cc], a, out_accum);
                }
                __syncthreads();
                for (int k = tid; k < 6 * T * T; k += kSplatThreads) scr[k] = 0ull;
                if (tid == 0) fr.tickets[slot] = 0;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Warp-per-item splat for tiles up to 32 px.  One warp owns every pixel of a square of at
// most 16 x 16 pixels (NR x NC blocks of 8 x 4 pixels, all in registers): a tile of up
// to 16 px, or one of the four quadrants of a larger tile, which are four separate work
// items over the same record list (binning with the larger tile keeps the scatter's
// open list slices within L2).  The warps of a CTA never wait on one another: in
// clustered data the density inside a tile is far from uniform, and with a tile's pixel
// rows shared out among several warps the busiest one set the pace.
// Per stage of 128 records (bulk copy into the warp's own double buffer, mbarrier
// completion with a bounded wait):
//   1. each lane takes 4 records: pixel box inside the square, and the rectangle of
//      blocks it covers; live records are counted per rectangle;
//   2. the live records are grouped by rectangle (warp-local counting sort), and their
//      colour (colormap, or the particle's emission in vector-colour scenes) and Gaussian
//      scale are computed, one record per lane;
//   3. for every rectangle present, one jump to straight-line code for that rectangle,
//      which runs over its records: each lane evaluates its pixel of every covered block
//      with the FP32 coverage rule and adds e * w to its registers.
// No atomics on pixels: a pixel has one owner.  Slices of a split tile add their partial
// sums into a scratch tile and the last one to finish writes the tile.

constexpr int kWarpsPerCta = 4;
constexpr int kWStage = 128;  // records per bulk copy, per warp

struct __align__(16) WRec {
    float X, Y, R2, kr;
    float er, eg, eb, pad;
};

struct __align__(16) WarpSmem {
    float4 buf[2][kWStage];      // staged records
    WRec dec[kWStage];           // decoded live records, grouped by rectangle
    int cnt[32];                 // live records per block rectangle
    unsigned char ord[kWStage];  // live records grouped by rectangle
    uint64_t bar[2];
};

template <int NR, int NC>
struct WarpShape {
    static constexpr int kRects = (NR * (NR + 1) / 2) * (NC * (NC + 1) / 2);
    static_assert(kRects <= 32, "one lane per block rectangle");
    // resident CTAs per SM, which caps the registers: below about 80 per thread the
    // compiler reloads record fields from shared memory instead of keeping them
    static constexpr int kMinCtas = NR * NC <= 2 ? 8 : 6;
};

// Index of the block range [a, b] among the n (n + 1) / 2 ranges of n blocks.
__host__ __device__ constexpr int range_id(int a, int b, int n) { return a * n - a * (a - 1) / 2 + (b - a); }

// Straight-line splat of one record over the block rectangle rows [R0, R1] x columns
// [C0, C1]: every lane evaluates its pixel of each block, uncovered pixels add zero.
template <int NR, int NC, int R0, int R1, int C0, int C1>
__device__ __forceinline__ void rect_splat(const float (&fx)[NC], const float (&fy)[NR], float (&ar)[NR][NC],
                                           float (&ag)[NR][NC], float (&ab)[NR][NC], const float4 &pa,
                                           const float4 &pb) {
    // dx^2 once per block column, dy^2 once per block row (same rounding as per pixel)
    float dx2[NC];
#pragma unroll
    for (int c = C0; c <= C1; ++c) {
        const float dx = __fsub_rn(fx[c], pa.x);
        dx2[c] = __fmul_rn(dx, dx);
    }
#pragma unroll
    for (int r = R0; r <= R1; ++r) {
        const float dy = __fsub_rn(fy[r], pa.y);
        const float dy2 = __fmul_rn(dy, dy);
#pragma unroll
        for (int c = C0; c <= C1; ++c) {
            const float d2 = __fadd_rn(dx2[c], dy2);
            const float w = ex2_fast(d2 * pa.w);
            // a += e * w only where d2 < R^2 (predicated: uncovered pixels add nothing)
            asm("{\n\t.reg .pred p;\n\t"
                "setp.lt.f32 p, %3, %4;\n\t"
                "@p fma.rn.f32 %0, %5, %8, %0;\n\t"
                "@p fma.rn.f32 %1, %6, %8, %1;\n\t"
                "@p fma.rn.f32 %2, %7, %8, %2;\n\t}"
                : "+f"(ar[r][c]), "+f"(ag[r][c]), "+f"(ab[r][c])
                : "f"(d2), "f"(pa.z), "f"(pb.x), "f"(pb.y), "f"(pb.z), "f"(w));
        }
    }
}

// All records of one block rectangle, taken from the grouped order: the jump to the
// rectangle's code is made once for the group.
template <int NR, int NC, int R0, int R1, int C0, int C1>
__device__ __forceinline__ void rect_run(const WarpSmem *ws, int j0, int n, const float (&fx)[NC],
                                         const float (&fy)[NR], float (&ar)[NR][NC], float (&ag)[NR][NC],
                                         float (&ab)[NR][NC]) {
    // not unrolled: 30 copies of an unrolled loop overflow the instruction cache
#pragma unroll 1
    for (int j = j0; j < j0 + n; ++j) {
        const float4 pa = *reinterpret_cast<const float4 *>(&ws->dec[j].X);
        const float4 pb = *reinterpret_cast<const float4 *>(&ws->dec[j].er);
        rect_splat<NR, NC, R0, R1, C0, C1>(fx, fy, ar, ag, ab, pa, pb);
    }
}

#define SPL_RUN(R0, R1, C0, C1)                                                               \
    case range_id(R0, R1, NR) * (NC * (NC + 1) / 2) + range_id(C0, C1, NC):                  \
        rect_run<NR, NC, R0, R1, C0, C1>(ws, j0, n, fx, fy, ar, ag, ab);                      \
        break;
#define SPL_RUNS4(C0, C1)                                                                      \
    SPL_RUN(0, 0, C0, C1) SPL_RUN(0, 1, C0, C1) SPL_RUN(0, 2, C0, C1) SPL_RUN(0, 3, C0, C1)     \
    SPL_RUN(1, 1, C0, C1) SPL_RUN(1, 2, C0, C1) SPL_RUN(1, 3, C0, C1) SPL_RUN(2, 2, C0, C1)     \
    SPL_RUN(2, 3, C0, C1) SPL_RUN(3, 3, C0, C1)

template <int NR, int NC>
__device__ __forceinline__ void run_dispatch(int id, const WarpSmem *ws, int j0, int n, const float (&fx)[NC],
                                             const float (&fy)[NR], float (&ar)[NR][NC], float (&ag)[NR][NC],
                                             float (&ab)[NR][NC]) {
    if constexpr (NR == 2 && NC == 1) {
        switch (id) {
            SPL_RUN(0, 0, 0, 0)
            SPL_RUN(0, 1, 0, 0)
            SPL_RUN(1, 1, 0, 0)
            default: break;
        }
    } else {
        static_assert(NR == 4 && NC == 2, "shapes: 8 x 8 and 16 x 16 pixels");
        switch (id) {
            SPL_RUNS4(0, 0)
            SPL_RUNS4(0, 1)
            SPL_RUNS4(1, 1)
            default: break;
        }
    }
}
#undef SPL_RUNS4
#undef SPL_RUN

// kViewScale: multiply every record's emission by a per-view, per-species scale (plans
// with a brightness sequence); a separate instance, so plain renders carry no extra code.
template <int NR, int NC, bool kViewScale, bool kEmit>
__global__ void __launch_bounds__(kWarpsPerCta * 32, (WarpShape<NR, NC>::kMinCtas))
    k_splat_warp(SceneDev sc, FrameDev fr, int *queue, float *out, int out_accum, int split) {
    if (fr.status[kStatOverflow] || fr.status[kStatTimeout]) return;  // no complete tile lists
    extern __shared__ __align__(16) unsigned char s_raw[];
    WarpSmem *ws = reinterpret_cast<WarpSmem *>(s_raw) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int nt = fr.n_tiles;
    const int N = fr.V * nt;
    const int S2 = split * split;
    const int total_items = (int)fr.sizes[kSizeItems] * S2;
    const int64_t K = fr.sizes[kSizeK];
    const ViewParams g0 = fr.views[0];
    const int T = g0.T, W = g0.W, H = g0.H, ntx = g0.ntx;
    const int sub = (T + split - 1) / split;  // edge of the square a warp owns
    const int lc = lane & 7, lr = lane >> 3;

    if (lane == 0) {
        mbar_init(&ws->bar[0], 1);
        mbar_init(&ws->bar[1], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t phase0 = 0, phase1 = 0;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(queue, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total_items) break;

        // item = (slice of a tile list, square of the tile); the squares of a slice are
        // consecutive items, so they run at once and share the slice's records in L2
        const int qs = item / S2, q = item - qs * S2;
        const int slice = fr.order ? __ldg(&fr.order[qs]) : qs;
        const int gt = find_tile(fr.item_off, N, slice);
        const int v = gt / nt, t = gt - v * nt;
        const int chunk = slice - fr.item_off[gt];
        const int arrivals = (fr.item_off[gt + 1] - fr.item_off[gt]) * S2;
        const int slot = fr.split_slot[gt];
        const float kexp = fr.views[v].kexp;
        const int tx = t % ntx, ty = t / ntx;
        const int qx = (q % split) * sub, qy = (q / split) * sub;
        const int px0 = tx * T + qx, py0 = ty * T + qy;
        const int tw = max(0, min(min(sub, T - qx), W - px0));
        const int th = max(0, min(min(sub, T - qy), H - py0));
        const int64_t seg1 = fr.offsets[gt + 1];
        const int64_t e0 = fr.offsets[gt] + (int64_t)chunk * K;
        const int nrec = (tw > 0 && th > 0) ? (int)(min(seg1, e0 + K) - e0) : 0;
        const int nst = (nrec + kWStage - 1) / kWStage;

        // this lane's pixels: (c * 8 + lc, r * 4 + lr) of the square; pixels outside it
        // get a centre no support reaches
        float fx[NC], fy[NR], ar[NR][NC], ag[NR][NC], ab[NR][NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) fx[c] = c * 8 + lc < tw ? (float)(px0 + c * 8 + lc) + 0.5f : kFar;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            fy[r] = r * 4 + lr < th ? (float)(py0 + r * 4 + lr) + 0.5f : kFar;
#pragma unroll
            for (int c = 0; c < NC; ++c) ar[r][c] = ag[r][c] = ab[r][c] = 0.0f;
        }

        if (lane == 0 && nrec > 0) {
            const int c0 = min(kWStage, nrec);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&ws->bar[0], (uint32_t)c0 * 16u);
            bulk_g2s(ws->buf[0], fr.lists + e0, (uint32_t)c0 * 16u, &ws->bar[0]);
        }
        for (int si = 0; si < nst; ++si) {
            const int cb = si & 1;
            if (lane == 0 && si + 1 < nst) {
                const int nb = (si + 1) & 1;
                const int cn = min(kWStage, nrec - (si + 1) * kWStage);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&ws->bar[nb], (uint32_t)cn * 16u);
                bulk_g2s(ws->buf[nb], fr.lists + e0 + (int64_t)(si + 1) * kWStage, (uint32_t)cn * 16u,
                         &ws->bar[nb]);
            }
            const bool ok = mbar_wait_bounded(&ws->bar[cb], cb ? phase1 : phase0, kWaitCycles);
            if (cb) phase1 ^= 1u; else phase0 ^= 1u;
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(&fr.status[kStatTimeout], 1);
                return;
            }
            const int cnt = min(kWStage, nrec - si * kWStage);
            const float4 *recs = ws->buf[cb];

            // ---- 1. pixel box and block rectangle of every record; count per rectangle
            ws->cnt[lane] = 0;
            __syncwarp();
            int rid[kWStage / 32], rrank[kWStage / 32];
#pragma unroll
            for (int q4 = 0; q4 < kWStage / 32; ++q4) {
                const int idx = q4 * 32 + lane;
                rid[q4] = -1;
                rrank[q4] = 0;
                if (idx < cnt) {
                    const float4 rec = recs[idx];
                    const float X = rec.x, Y = rec.y, R = rec.z;
                    // tight pixel range of the support inside the square; eps exceeds the
                    // FP32 rounding of X +- R at any position, so no covered pixel is lost
                    const float eps = 1e-3f + 2e-6f * (fabsf(X) + fabsf(Y) + R);
                    const int ilo = max(0, (int)ceilf(clampf(X - R - 0.5f - eps, px0 - 1.0f, (float)(px0 + tw))) - px0);
                    const int ihi = min(tw - 1, (int)floorf(clampf(X + R - 0.5f + eps, px0 - 1.0f, (float)(px0 + tw))) - px0);
                    const int jlo = max(0, (int)ceilf(clampf(Y - R - 0.5f - eps, py0 - 1.0f, (float)(py0 + th))) - py0);
                    const int jhi = min(th - 1, (int)floorf(clampf(Y + R - 0.5f + eps, py0 - 1.0f, (float)(py0 + th))) - py0);
                    if (ilo <= ihi && jlo <= jhi)
                        rid[q4] = range_id(jlo >> 2, jhi >> 2, NR) * (NC * (NC + 1) / 2) +
                                  range_id(ilo >> 3, ihi >> 3, NC);
                }
                // rank among the stage's records of the same rectangle, in record order
                // (lanes with equal rectangle ids, found bit by bit with ballots)
                const uint32_t peers = warp_peers<6>((uint32_t)(rid[q4] + 1));
                const int leader = __ffs(peers) - 1;
                int before = 0;
                if (rid[q4] >= 0 && lane == leader) {
                    before = ws->cnt[rid[q4]];
                    ws->cnt[rid[q4]] = before + __popc(peers);
                }
                before = __shfl_sync(0xffffffffu, before, leader);
                rrank[q4] = before + __popc(peers & ((1u << lane) - 1u));
                __syncwarp();
            }
            __syncwarp();
            // ---- 2. group the live records by rectangle (lane = rectangle)
            const int c = ws->cnt[lane];
            const int incl = warp_incl_scan_i(c);
            const int base = incl - c;
            const int nlive = __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
            for (int q4 = 0; q4 < kWStage / 32; ++q4) {
                const int b = __shfl_sync(0xffffffffu, base, rid[q4] < 0 ? 0 : rid[q4]);
                if (rid[q4] >= 0) ws->ord[b + rrank[q4]] = (unsigned char)(q4 * 32 + lane);
            }
            __syncwarp();
            // colour and Gaussian scale of the live records only, one per lane
            for (int j = lane; j < nlive; j += 32) {
                const int k = ws->ord[j];
                const float4 rec = recs[k];
                const float R = rec.z;
                const uint32_t code = __float_as_uint(rec.w);
                int type;
                float3 e;
                if constexpr (kEmit) {
                    const float4 em = __ldg(&sc.emit[code]);  // the code is the particle index
                    type = __float_as_int(em.w);
                    e = make_float3(em.x, em.y, em.z);
                } else {
                    type = (int)(code >> 24);
                    const float It = fminf((float)(code & kCodeMax) * (1.0f / (float)kCodeMax), 1.0f);
                    // the view's colormap in a plan with per-view sequences, else the scene's
                    const float4 *lut = sc.lut;
                    int len, off;
                    if constexpr (kViewScale) {
                        const int vi = v * sc.n_types + type;
                        lut = fr.vlut;
                        len = __ldg(&fr.vlut_len[vi]);
                        off = __ldg(&fr.vlut_off[vi]);
                    } else {
                        len = __ldg(&sc.lut_len[type]);
                        off = __ldg(&sc.lut_off[type]);
                    }
                    const float f = It * (float)(len - 1);
                    const int kk = min((int)f, len - 2);
                    const float tau = f - (float)kk;
                    const float4 c0 = __ldg(&lut[off + kk]);
                    const float4 c1 = __ldg(&lut[off + kk + 1]);
                    e = make_float3((1.0f - tau) * c0.x + tau * c1.x, (1.0f - tau) * c0.y + tau * c1.y,
                                    (1.0f - tau) * c0.z + tau * c1.z);
                }
                const float R2 = __fmul_rn(R, R);
                float vs = 1.0f;
                if constexpr (kViewScale) vs = __ldg(&fr.vscale[v * sc.n_types + type]);
                float4 *d = reinterpret_cast<float4 *>(&ws->dec[j]);  // in grouped order
                d[0] = make_float4(rec.x, rec.y, R2, __fdividef(kexp, R2));
                d[1] = make_float4(e.x * vs, e.y * vs, e.z * vs, 0.0f);
            }
            __syncwarp();
            // ---- 3. one jump per rectangle present, then its records
            uint32_t present = __ballot_sync(0xffffffffu, c > 0);
            while (present) {
                const int id = __ffs(present) - 1;
                present &= present - 1;
                const int j0 = __shfl_sync(0xffffffffu, base, id);
                const int n = __shfl_sync(0xffffffffu, c, id);
                run_dispatch<NR, NC>(id, ws, j0, n, fx, fy, ar, ag, ab);
            }
            __syncwarp();
        }

        // epilogue: final transform of this lane's pixels, or merge of a split tile
        float *o = out + (int64_t)v * H * W * 3;
        if (slot < 0) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (r * 4 + lr >= th) continue;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    if (cc * 8 + lc >= tw) continue;
                    float *p = o + ((int64_t)(py0 + r * 4 + lr) * W + px0 + cc * 8 + lc) * 3;
                    put_pixel(p, ar[r][cc], out_accum);
                    put_pixel(p + 1, ag[r][cc], out_accum);
                    put_pixel(p + 2, ab[r][cc], out_accum);
                }
            }
        } else {
            unsigned long long *scr = fr.scratch + (int64_t)slot * 6 * T * T;
            // the lane's sums go through the warp's (now idle) decode area so that one
            // loop, not an unrolled copy per pixel, adds them: the splat's straight-line
            // code already fills the instruction cache
            float *park = reinterpret_cast<float *>(ws->dec) + lane;  // [NR * NC * 3][32]
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const int k = 3 * (r * NC + cc);
                    park[32 * k] = ar[r][cc];
                    park[32 * (k + 1)] = ag[r][cc];
                    park[32 * (k + 2)] = ab[r][cc];
                }
#pragma unroll 1
            for (int k = 0; k < 3 * NR * NC; ++k) {
                const int ch = k % 3, blk = k / 3, r = blk / NC, cc = blk - r * NC;
                if (r * 4 + lr >= th || cc * 8 + lc >= tw) continue;
                const int pix = (qy + r * 4 + lr) * T + qx + cc * 8 + lc;
                fix_add(&scr[2 * (ch * T * T + pix)], park[32 * k]);
            }
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = (atomicAdd(&fr.tickets[slot], 1) == arrivals - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                // the whole tile, from the scratch every square of every slice added into
                __threadfence();
                const int TW = min(T, W - tx * T), TH = min(T, H - ty * T);
                const int rowlen = 3 * TW;
                float *ot = o + ((int64_t)ty * T * W + (int64_t)tx * T) * 3;
                for (int k = lane; k < TH * rowlen; k += 32) {
                    const int rr = k / rowlen, c3 = k - rr * rowlen;
                    const int col = c3 / 3, ch = c3 - col * 3;
                    const float a = fix_value(&scr[2 * (ch * T * T + rr * T + col)]);
                    put_pixel(&ot[(int64_t)rr * W * 3 + c3], a, out_accum);
                }
                __syncwarp();
                for (int k = lane; k < 6 * T * T; k += 32) scr[k] = 0ull;
                if (lane == 0) fr.tickets[slot] = 0;
            }
        }
        __syncwarp();
    }
}

typedef void (*SplatFn)(SceneDev, FrameDev, int *, float *, int);
typedef void (*WarpSplatFn)(SceneDev, FrameDev, int *, float *, int, int);

// Tiles up to 32 px: warp per square of up to 16 px (a tile above 16 px is split into
// four squares); larger tiles: CTA per item.
constexpr int kWarpTileMax = 32;
static bool warp_kernel(int T) { return T <= kWarpTileMax; }
int splat_split(int T) { return T > 16 && warp_kernel(T) ? 2 : 1; }

static WarpSplatFn warp_fn(int T, bool scaled = false, bool emit = false) {
    if (emit) {
        if (scaled) return T <= 8 ? k_splat_warp<2, 1, true, true> : k_splat_warp<4, 2, true, true>;
        return T <= 8 ? k_splat_warp<2, 1, false, true> : k_splat_warp<4, 2, false, true>;
    }
    if (scaled) return T <= 8 ? k_splat_warp<2, 1, true, false> : k_splat_warp<4, 2, true, false>;
    return T <= 8 ? k_splat_warp<2, 1, false, false> : k_splat_warp<4, 2, false, false>;
}

static SplatFn cta_fn(int T) {
    switch (block_cols(T)) {
        case 5: return k_splat<2, 5>;
        case 6: return k_splat<2, 6>;
        case 7: return k_splat<2, 7>;
        default: return k_splat<2, 8>;
    }
}

static const void *splat_kernel(int T) { return warp_kernel(T) ? (const void *)warp_fn(T) : (const void *)cta_fn(T); }

static size_t splat_smem(int T) { return warp_kernel(T) ? sizeof(WarpSmem) * kWarpsPerCta : splat_smem_bytes(T); }
static int splat_cta_threads(int T) { return warp_kernel(T) ? kWarpsPerCta * 32 : kSplatThreads; }

int splat_blocks_per_sm(int T) {
    const size_t smem = splat_smem(T);
    const void *fn = splat_kernel(T);
    if (ensure_smem_limit(fn, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, splat_cta_threads(T), smem) != cudaSuccess) return 0;
    return nb;
}

int splat_workers_per_sm(int T) { return splat_blocks_per_sm(T) * (warp_kernel(T) ? kWarpsPerCta : 1); }

// k_item_order: one CTA.  The splat's work items (tile-list slices) ordered by record count,
// largest first, so that the items taken last by the workers are the short ones and the
// kernel does not end waiting for a few long slices started late.  Slices fall into
// kOrderBins bins of equal width up to K (the slice length of a split tile); within a bin
// the order is that of the atomic cursors.  Each item writes its own tile, or adds into
// the exact accumulators of a split tile, so images do not depend on the order.
constexpr int kOrderBins = 64;

__global__ void __launch_bounds__(1024) k_item_order(FrameDev fr) {
    __shared__ int s_cnt[kOrderBins];
    if (fr.status[kStatOverflow]) return;
    const int N = fr.V * fr.n_tiles;
    const long long K = fr.sizes[kSizeK];
    auto bin_of = [&](long long size) -> int {
        return (int)min((long long)(kOrderBins - 1), size * kOrderBins / (K + 1));
    };
    for (int b = threadIdx.x; b < kOrderBins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    // (1) slices per size bin: every slice of a split tile holds K records but the last
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int i0 = fr.item_off[t], n = fr.item_off[t + 1] - i0;
        const long long c = fr.counts[t];
        if (n > 1) atomicAdd(&s_cnt[bin_of(K)], n - 1);
        atomicAdd(&s_cnt[bin_of(c - K * (n - 1))], 1);
    }
    __syncthreads();
    // (2) bin starts, the largest bin first
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = kOrderBins - 1; b >= 0; --b) {
            const int c = s_cnt[b];
            s_cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    // (3) every slice at its bin's next place
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int i0 = fr.item_off[t], n = fr.item_off[t + 1] - i0;
        const long long c = fr.counts[t];
        if (n > 1) {
            const int p = atomicAdd(&s_cnt[bin_of(K)], n - 1);
            for (int s = 0; s < n - 1; ++s) fr.order[p + s] = i0 + s;
        }
        fr.order[atomicAdd(&s_cnt[bin_of(c - K * (n - 1))], 1)] = i0 + n - 1;
    }
}

cudaError_t launch_item_order(const FrameDev &fr, cudaStream_t st) {
    if (!fr.order) return cudaSuccess;
    k_item_order<<<1, 1024, 0, st>>>(fr);
    return cudaGetLastError();
}

cudaError_t launch_splat(const SceneDev &sc, const FrameDev &fr, int *queue, float *out, int out_accum,
                         int grid, cudaStream_t st) {
    cudaError_t e = launch_item_order(fr, st);
    if (e != cudaSuccess) return e;
    const size_t smem = splat_smem(fr.T);
    const bool scaled = fr.vscale != nullptr, emit = sc.emit != nullptr;
    cudaError_t err = ensure_smem_limit(
        warp_kernel(fr.T) ? (const void *)warp_fn(fr.T, scaled, emit) : splat_kernel(fr.T), smem);
    if (err != cudaSuccess) return err;
    if (warp_kernel(fr.T))
        warp_fn(fr.T, scaled, emit)<<<grid, splat_cta_threads(fr.T), smem, st>>>(sc, fr, queue, out, out_accum,
                                                                                   splat_split(fr.T));
    else
        cta_fn(fr.T)<<<grid, splat_cta_threads(fr.T), smem, st>>>(sc, fr, queue, out, out_accum);
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
