// Depth-ordered splat: radiative transfer with absorption different from emission.
//
// Section 2.1 renders by solving the radiative-transfer equation along each line of
// sight.  With absorption A equal to emission E every particle's update commutes and the
// image is 1 - exp(-a) of a plain sum; with A = s_t E for species t (s_t >= 0) it does
// not, and the particles must be applied in depth order, farthest first, from a black
// background:
//     I <- a I + b,   a = exp(-A w),   b = (E / A)(1 - a) = (1 - a) / s_t   (I + E w if s_t = 0)
// per pixel and channel, w the particle's Gaussian weight there.  The tile lists reach
// this kernel far to near, particles of exactly equal depth in index order: the particles
// are sorted by depth (stably, from index order), their records are written out in that
// order, and a stable sort by tile id groups them (depth-ordered binning).
//
// Layout as the additive warp kernel: one warp owns a square of up to 16 x 16 pixels (a
// tile, or a quarter of a larger one), blocks of 8 x 4 pixels, one pixel of each block
// per lane, state in registers.  Records are taken 32 at a time (decoded one per lane)
// and applied strictly in list order.  Each lane keeps, per pixel and channel, the affine
// map of the records applied so far, I_out = alpha I_in + beta: a tile that is not split
// writes beta; the slices of a split tile store their maps, and the last slice to finish
// composes them far to near.
#include "splotch_internal.cuh"

namespace spl {

constexpr int kOWarps = 4;     // warps per CTA
constexpr int kOStage = 128;   // records per bulk copy, per warp
constexpr int kONR = 4, kONC = 2;  // block rows x block columns of a 16 x 16 square
constexpr float kOFar = 1e30f;

struct __align__(16) ORec {
    float X, Y, R2, kr;       // centre, support^2, Gaussian scale (w = 2^(d^2 kr))
    float kxr, kxg, kxb, inv_s;  // A = s E per channel (x = A w); 1 / s (0 when s = 0)
    float er, eg, eb;         // emission E
    uint32_t mask;            // blocks (r * kONC + c) the record's box overlaps
};

struct __align__(16) OWarpSmem {
    float4 buf[2][kOStage];
    ORec dec[32];
    uint64_t bar[2];
};

__device__ __forceinline__ int find_tile_o(const int *__restrict__ item_off, int N, int item) {
    int a = 0, b = N - 1;  // last gt with item_off[gt] <= item
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (__ldg(&item_off[m]) <= item) a = m; else b = m - 1;
    }
    return a;
}

// A record whose largest x = s E w (w <= 1) is small takes a series path: with
// phi(x) = (1 - exp(-x)) / x = sum_k (-x)^k / (k + 1)!, a = 1 - x phi and b = E w phi, no
// exponential per channel.  phi to degree 2 where x <= kSeries2Max (next term x^3 / 24
// <= 1.5e-7 relative), to degree 5 where x <= kSeries5Max (x^6 / 7! <= 5e-8).
constexpr float kSeries2Max = 0.015f, kSeries5Max = 0.25f;
constexpr uint32_t kSeries5Flag = 1u << 31, kSeries2Flag = 1u << 30;  // in the record's block mask

// Per-lane state: the lane's pixels of block rows 2p and 2p + 1 (same column block c)
// are held as the two halves of a float2, so that one packed FP32x2 instruction updates
// both; a pair is computed when either of its two blocks is in the record's mask (a block
// outside the record's box has no covered pixel, and an uncovered pixel's update is the
// identity a = 1, b = 0).
constexpr int kONP = kONR / 2;  // row pairs

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Apply one record: per pixel and channel I <- a I + b, and the slice map's alpha <- a alpha.
template <int kDeg>  // 2 or 5: series of that degree; 0: exponential
__device__ __forceinline__ void apply_record(const float4 &pa, const float4 &pk, const float4 &pe, uint32_t m,
                                             const float (&fx)[kONC], const float2 (&fy)[kONP],
                                             float2 (&al)[kONP][kONC][3], float2 (&be)[kONP][kONC][3]) {
#pragma unroll
    for (int q = 0; q < kONP; ++q) {
        // blocks (2q, c) and (2q + 1, c), c = 0, 1: mask bits 4q .. 4q + 3
        if (!(m & (0xFu << (4 * q)))) continue;
        const float2 dy = __fadd2_rn(fy[q], f2(-pa.y));
        const float2 dy2 = __fmul2_rn(dy, dy);
#pragma unroll
        for (int c = 0; c < kONC; ++c) {
            if (!(m & ((1u << c) | (1u << (kONC + c))) << (4 * q))) continue;
            const float dx = __fsub_rn(fx[c], pa.x);
            const float2 d2 = __fadd2_rn(f2(__fmul_rn(dx, dx)), dy2);
            const float2 e = __fmul2_rn(d2, f2(pa.w));
            float2 w = make_float2(ex2_fast(e.x), ex2_fast(e.y));
            w.x = d2.x < pa.z ? w.x : 0.0f;  // uncovered: a = 1, b = 0
            w.y = d2.y < pa.z ? w.y : 0.0f;
            const float kx[3] = {pk.x, pk.y, pk.z}, E[3] = {pe.x, pe.y, pe.z};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float2 x = __fmul2_rn(f2(kx[ch]), w);
                float2 a, b;
                if (kDeg > 0) {
                    float2 phi;
                    if (kDeg == 5) {
                        phi = __ffma2_rn(x, f2(-1.0f / 720.0f), f2(1.0f / 120.0f));
                        phi = __ffma2_rn(x, phi, f2(-1.0f / 24.0f));
                        phi = __ffma2_rn(x, phi, f2(1.0f / 6.0f));
                    } else {
                        phi = f2(1.0f / 6.0f);
                    }
                    phi = __ffma2_rn(x, phi, f2(-0.5f));
                    phi = __ffma2_rn(x, phi, f2(1.0f));
                    a = __ffma2_rn(make_float2(-x.x, -x.y), phi, f2(1.0f));
                    b = __fmul2_rn(__fmul2_rn(f2(E[ch]), w), phi);
                } else {
                    // a = exp(-x), b = (1 - a) / s.  Where x is small, 1 - a in FP32 would
                    // cancel most digits: there phi to degree 2 (next term x^3 / 24), so
                    // a = 1 - x phi and b = E w phi (also the s = 0 case)
                    const float2 phi = __ffma2_rn(x, __ffma2_rn(x, f2(1.0f / 6.0f), f2(-0.5f)), f2(1.0f));
                    const float2 as = __ffma2_rn(make_float2(-x.x, -x.y), phi, f2(1.0f));
                    const float2 bs = __fmul2_rn(__fmul2_rn(f2(E[ch]), w), phi);
                    const float2 ag = make_float2(ex2_fast(x.x * -kLog2e), ex2_fast(x.y * -kLog2e));
                    const float2 bg = __ffma2_rn(make_float2(-ag.x, -ag.y), f2(pk.w), f2(pk.w));
                    a = make_float2(x.x < 0.015f ? as.x : ag.x, x.y < 0.015f ? as.y : ag.y);
                    b = make_float2(x.x < 0.015f ? bs.x : bg.x, x.y < 0.015f ? bs.y : bg.y);
                }
                al[q][c][ch] = __fmul2_rn(al[q][c][ch], a);
                be[q][c][ch] = __ffma2_rn(a, be[q][c][ch], b);
            }
        }
    }
}

// Element (block row r, column block c, channel ch) of a lane's paired state.
#define OSTATE(arr, r, c, ch) (((r) & 1) ? arr[(r) >> 1][c][ch].y : arr[(r) >> 1][c][ch].x)

__global__ void __launch_bounds__(kOWarps * 32, 4)
    k_splat_ordered(SceneDev sc, FrameDev fr, int *queue, float *out, int split,
                    const float *__restrict__ absorb, float *ord_scratch, int map_out) {
    if (fr.status[kStatOverflow]) return;
    extern __shared__ __align__(16) unsigned char s_raw[];
    OWarpSmem *ws = reinterpret_cast<OWarpSmem *>(s_raw) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int nt = fr.n_tiles;
    const int N = fr.V * nt;
    const int S2 = split * split;
    const int total_items = (int)fr.sizes[kSizeItems] * S2;
    const int64_t K = fr.sizes[kSizeK];
    const ViewParams g0 = fr.views[0];
    const int T = g0.T, W = g0.W, H = g0.H, ntx = g0.ntx;
    const int sub = (T + split - 1) / split;
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

        const int qs = item / S2, q = item - qs * S2;
        const int slice = fr.order ? __ldg(&fr.order[qs]) : qs;  // largest slices first
        const int gt = find_tile_o(fr.item_off, N, slice);
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
        const int nst = (nrec + kOStage - 1) / kOStage;

        float fx[kONC];
        float2 fy[kONP], al[kONP][kONC][3], be[kONP][kONC][3];
#pragma unroll
        for (int c = 0; c < kONC; ++c) fx[c] = c * 8 + lc < tw ? (float)(px0 + c * 8 + lc) + 0.5f : kOFar;
#pragma unroll
        for (int q = 0; q < kONP; ++q) {
            const int r0 = 2 * q, r1 = 2 * q + 1;
            fy[q] = make_float2(r0 * 4 + lr < th ? (float)(py0 + r0 * 4 + lr) + 0.5f : kOFar,
                                r1 * 4 + lr < th ? (float)(py0 + r1 * 4 + lr) + 0.5f : kOFar);
#pragma unroll
            for (int c = 0; c < kONC; ++c)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) al[q][c][ch] = f2(1.0f), be[q][c][ch] = f2(0.0f);
        }

        if (lane == 0 && nrec > 0) {
            const int c0 = min(kOStage, nrec);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&ws->bar[0], (uint32_t)c0 * 16u);
            bulk_g2s(ws->buf[0], fr.lists + e0, (uint32_t)c0 * 16u, &ws->bar[0]);
        }
        for (int si = 0; si < nst; ++si) {
            const int cb = si & 1;
            if (lane == 0 && si + 1 < nst) {
                const int nb = (si + 1) & 1;
                const int cn = min(kOStage, nrec - (si + 1) * kOStage);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&ws->bar[nb], (uint32_t)cn * 16u);
                bulk_g2s(ws->buf[nb], fr.lists + e0 + (int64_t)(si + 1) * kOStage, (uint32_t)cn * 16u,
                         &ws->bar[nb]);
            }
            const bool ok = mbar_wait_bounded(&ws->bar[cb], cb ? phase1 : phase0, kWaitCycles);
            if (cb) phase1 ^= 1u; else phase0 ^= 1u;
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(&fr.status[kStatTimeout], 1);
                return;
            }
            const int cnt = min(kOStage, nrec - si * kOStage);
            for (int g = 0; g < cnt; g += 32) {
                // ---- decode: one record per lane
                uint32_t mask = 0;
                if (g + lane < cnt) {
                    const float4 rec = ws->buf[cb][g + lane];
                    const float X = rec.x, Y = rec.y, R = rec.z;
                    const uint32_t code = __float_as_uint(rec.w);
                    const float eps = 1e-3f + 2e-6f * (fabsf(X) + fabsf(Y) + R);
                    const int ilo = max(0, (int)ceilf(clampf(X - R - 0.5f - eps, px0 - 1.0f, (float)(px0 + tw))) - px0);
                    const int ihi = min(tw - 1, (int)floorf(clampf(X + R - 0.5f + eps, px0 - 1.0f, (float)(px0 + tw))) - px0);
                    const int jlo = max(0, (int)ceilf(clampf(Y - R - 0.5f - eps, py0 - 1.0f, (float)(py0 + th))) - py0);
                    const int jhi = min(th - 1, (int)floorf(clampf(Y + R - 0.5f + eps, py0 - 1.0f, (float)(py0 + th))) - py0);
                    if (ilo <= ihi && jlo <= jhi) {
                        const uint32_t cm = (2u << (ihi >> 3)) - (1u << (ilo >> 3));
                        for (int r = jlo >> 2; r <= (jhi >> 2); ++r) mask |= cm << (r * kONC);
                        int type;
                        float er, eg, eb;
                        if (sc.emit) {
                            const float4 em = __ldg(&sc.emit[code]);  // the code is the particle index
                            type = __float_as_int(em.w);
                            er = em.x, eg = em.y, eb = em.z;
                        } else {
                            type = (int)(code >> 24);
                            const float It = fminf((float)(code & kCodeMax) * (1.0f / (float)kCodeMax), 1.0f);
                            const int len = __ldg(&sc.lut_len[type]);
                            const float f = It * (float)(len - 1);
                            const int kk = min((int)f, len - 2);
                            const float tau = f - (float)kk;
                            const int lo = __ldg(&sc.lut_off[type]) + kk;
                            const float4 c0 = __ldg(&sc.lut[lo]);
                            const float4 c1 = __ldg(&sc.lut[lo + 1]);
                            er = (1.0f - tau) * c0.x + tau * c1.x;
                            eg = (1.0f - tau) * c0.y + tau * c1.y;
                            eb = (1.0f - tau) * c0.z + tau * c1.z;
                        }
                        const float s = __ldg(&absorb[type]);
                        const float R2 = __fmul_rn(R, R);
                        float4 *d = reinterpret_cast<float4 *>(&ws->dec[lane]);
                        d[0] = make_float4(X, Y, R2, __fdividef(kexp, R2));
                        d[1] = make_float4(s * er, s * eg, s * eb, s > 0.0f ? 1.0f / s : 0.0f);
                        const float xmax = s * fmaxf(fabsf(er), fmaxf(fabsf(eg), fabsf(eb)));
                        const uint32_t path = xmax <= kSeries2Max ? kSeries2Flag : (xmax <= kSeries5Max ? kSeries5Flag : 0u);
                        d[2] = make_float4(er, eg, eb, __uint_as_float(mask | path));
                    }
                }
                uint32_t live = __ballot_sync(0xffffffffu, mask != 0);
                __syncwarp();
                // ---- apply the live records in list order (far to near)
                while (live) {
                    const int k = __ffs(live) - 1;
                    live &= live - 1;
                    const float4 pa = *reinterpret_cast<const float4 *>(&ws->dec[k].X);
                    const float4 pk = *reinterpret_cast<const float4 *>(&ws->dec[k].kxr);
                    const float4 pe = *reinterpret_cast<const float4 *>(&ws->dec[k].er);
                    const uint32_t m = __float_as_uint(pe.w);
                    if (m & kSeries2Flag)
                        apply_record<2>(pa, pk, pe, m, fx, fy, al, be);
                    else if (m & kSeries5Flag)
                        apply_record<5>(pa, pk, pe, m, fx, fy, al, be);
                    else
                        apply_record<0>(pa, pk, pe, m, fx, fy, al, be);
                }
                __syncwarp();
            }
        }

        // epilogue: a whole tile writes I = beta (black background), or with map_out the
        // map (alpha rgb, beta rgb); a slice of a split tile stores its map, and the last
        // slice composes the tile far to near
        const int oc = map_out ? 6 : 3;  // floats per pixel
        float *o = out + (int64_t)v * H * W * oc;
        if (slot < 0) {
#pragma unroll
            for (int r = 0; r < kONR; ++r) {
                if (r * 4 + lr >= th) continue;
#pragma unroll
                for (int c = 0; c < kONC; ++c) {
                    if (c * 8 + lc >= tw) continue;
                    float *p = o + ((int64_t)(py0 + r * 4 + lr) * W + px0 + c * 8 + lc) * oc;
                    if (map_out) {
                        p[0] = OSTATE(al, r, c, 0);
                        p[1] = OSTATE(al, r, c, 1);
                        p[2] = OSTATE(al, r, c, 2);
                        p += 3;
                    }
                    p[0] = OSTATE(be, r, c, 0);
                    p[1] = OSTATE(be, r, c, 1);
                    p[2] = OSTATE(be, r, c, 2);
                }
            }
        } else {
            float *map = ord_scratch + (int64_t)slice * 6 * T * T;  // [alpha r g b, beta r g b][T][T]
#pragma unroll
            for (int r = 0; r < kONR; ++r) {
                if (r * 4 + lr >= th) continue;
#pragma unroll
                for (int c = 0; c < kONC; ++c) {
                    if (c * 8 + lc >= tw) continue;
                    const int pix = (qy + r * 4 + lr) * T + qx + c * 8 + lc;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        map[ch * T * T + pix] = OSTATE(al, r, c, ch);
                        map[(3 + ch) * T * T + pix] = OSTATE(be, r, c, ch);
                    }
                }
            }
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = (atomicAdd(&fr.tickets[slot], 1) == arrivals - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                const int TW = min(T, W - tx * T), TH = min(T, H - ty * T);
                const int s0 = fr.item_off[gt], s1 = fr.item_off[gt + 1];
                float *ot = o + ((int64_t)ty * T * W + (int64_t)tx * T) * oc;
                for (int k = lane; k < TH * TW * 3; k += 32) {
                    const int pix3 = k / 3, ch = k - pix3 * 3;
                    const int rr = pix3 / TW, col = pix3 - rr * TW;
                    const int pix = rr * T + col;
                    float A = 1.0f, I = 0.0f;
                    for (int sl = s0; sl < s1; ++sl) {
                        const float *ms = ord_scratch + (int64_t)sl * 6 * T * T;
                        const float a = __ldcg(&ms[ch * T * T + pix]);
                        I = fmaf(a, I, __ldcg(&ms[(3 + ch) * T * T + pix]));
                        A *= a;
                    }
                    float *q = ot + (int64_t)rr * W * oc + col * oc;
                    if (map_out) {
                        q[ch] = A;
                        q[3 + ch] = I;
                    } else {
                        q[ch] = I;
                    }
                }
                if (lane == 0) fr.tickets[slot] = 0;
            }
        }
        __syncwarp();
    }
}

__global__ void k_gather_records(const float4 *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                                 float4 *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

cudaError_t launch_gather_records(const float4 *src, const uint32_t *idx, int64_t n, float4 *dst, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_gather_records<<<grid_for(n), 256, 0, st>>>(src, idx, n, dst);
    return cudaGetLastError();
}

int ordered_split(int T) { return T > 16 ? 2 : 1; }

static size_t ordered_smem() { return sizeof(OWarpSmem) * kOWarps; }

int ordered_ctas_per_sm() {
    if (ensure_smem_limit((const void *)k_splat_ordered, ordered_smem()) != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_splat_ordered, kOWarps * 32, ordered_smem()) !=
        cudaSuccess)
        return 1;
    return std::max(1, nb);
}

int ordered_workers_per_sm() { return ordered_ctas_per_sm() * kOWarps; }

// Composition of depth-slab maps (Section 2.1: the transfer along a line of sight takes
// the farther material first; Section 4.2.2: tasks render their particles independently).
// maps: n arrays of `pixels` x 6 floats, farthest first, each pixel (alpha rgb, beta rgb)
// of I_out = alpha I_in + beta.  Composing far to near: beta <- alpha_k beta + beta_k,
// alpha <- alpha_k alpha.  One thread per (pixel, channel); the result's beta is the
// frame from a black background.
__global__ void k_compose_maps(const float *__restrict__ maps, int n, int64_t pixels, float *__restrict__ out) {
    const int64_t count = pixels * 3, stride = pixels * 6;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = j / 3;
        const int64_t ia = p * 6 + (j - p * 3), ib = ia + 3;
        float a = maps[ia], b = maps[ib];
        for (int k = 1; k < n; ++k) {
            const float ak = maps[k * stride + ia], bk = maps[k * stride + ib];
            b = __fmaf_rn(ak, b, bk);
            a = __fmul_rn(ak, a);
        }
        out[ia] = a;
        out[ib] = b;
    }
}

cudaError_t launch_compose_maps(const float *maps, int n, int64_t pixels, float *out, cudaStream_t st) {
    if (pixels <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((pixels * 3 + 255) / 256, 152 * 16);
    k_compose_maps<<<(int)blocks, 256, 0, st>>>(maps, n, pixels, out);
    return cudaGetLastError();
}

cudaError_t launch_splat_ordered(const SceneDev &sc, const FrameDev &fr, int *queue, float *out,
                                 const float *absorb, float *ord_scratch, int map_out, int grid, cudaStream_t st) {
    cudaError_t err = ensure_smem_limit((const void *)k_splat_ordered, ordered_smem());
    if (err != cudaSuccess) return err;
    if ((err = launch_item_order(fr, st)) != cudaSuccess) return err;
    k_splat_ordered<<<grid, kOWarps * 32, ordered_smem(), st>>>(sc, fr, queue, out, ordered_split(fr.T), absorb,
                                                                ord_scratch, map_out);
    return cudaGetLastError();
}

}  // namespace spl
