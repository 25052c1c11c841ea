// Host runtime of the Splotch C ABI (include/splotch.h): scene residency, camera
// composition, frame workspace sizing and the launch sequence count -> scan ->
// scatter -> splat, the debug hooks and the pre-sized multi-view plan.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "splotch.h"
#include "splotch_internal.cuh"

using namespace spl;

// -----------------------------------------------------------------------------------------
// errors

static thread_local char g_err[512];

static splotch_status fail(splotch_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(SPLOTCH_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                        __FILE__, __LINE__);                                                    \
    } while (0)

extern "C" const char *splotch_status_string(splotch_status s) {
    switch (s) {
    case SPLOTCH_OK: return "ok";
    case SPLOTCH_ERR_INVALID_ARG: return "invalid argument";
    case SPLOTCH_ERR_OOM: return "out of device memory";
    case SPLOTCH_ERR_CUDA: return "CUDA error";
    case SPLOTCH_ERR_CAPACITY: return "pre-sized capacity exceeded";
    case SPLOTCH_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPLOTCH_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

extern "C" const char *splotch_last_error(void) { return g_err; }

// -----------------------------------------------------------------------------------------
// device memory: caller callbacks, or one stream-ordered pool per device

static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;

static cudaMemPool_t device_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

struct Mem {
    splotch_allocator a{};
    int dev = 0;
    bool custom() const { return a.alloc != nullptr; }
    void *alloc(size_t bytes, cudaStream_t st) const {
        if (bytes == 0) bytes = 256;
        if (custom()) return a.alloc(a.ctx, bytes, (void *)st);
        cudaMemPool_t pool = device_pool(dev);
        if (!pool) return nullptr;
        void *p = nullptr;
        if (cudaMallocFromPoolAsync(&p, bytes, pool, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void release(void *p, cudaStream_t st) const {
        if (!p) return;
        if (custom()) {
            if (a.free) a.free(a.ctx, p, (void *)st);
        } else {
            cudaFreeAsync(p, st);
        }
    }
};

static inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Sub-buffers carved from one allocation.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    }
};

static int sm_count(int dev) {
    static std::mutex mu;
    static std::vector<int> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (!cache[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

// small pinned host buffer per thread for size / status read-back
struct HostBox {
    int64_t *p = nullptr;
    ~HostBox() {
        if (p) cudaFreeHost(p);
    }
};
static thread_local HostBox g_box;
static int64_t *host_box() {
    if (!g_box.p) {
        if (cudaMallocHost((void **)&g_box.p, 64 * sizeof(int64_t)) != cudaSuccess) {
            cudaGetLastError();
            g_box.p = nullptr;
        }
    }
    return g_box.p;
}

// per-thread kernel timing of the last SPLOTCH_TIMING render
struct Timing {
    cudaEvent_t ev[6] = {};
    bool have = false;
    double ms[4] = {0, 0, 0, 0};
    int64_t counts[3] = {0, 0, 0};
    ~Timing() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    bool init() {
        for (auto &e : ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
        return true;
    }
};
static thread_local Timing g_timing;

extern "C" splotch_status splotch_last_timing(double ms[4], int64_t counts[3]) {
    if (!g_timing.have) return fail(SPLOTCH_ERR_INVALID_ARG, "no timed render on this thread");
    if (ms)
        for (int k = 0; k < 4; ++k) ms[k] = g_timing.ms[k];
    if (counts)
        for (int k = 0; k < 3; ++k) counts[k] = g_timing.counts[k];
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// scene

struct splotch_scene {
    int dev = 0;
    int64_t n = 0, n_pad = 0;
    int n_types = 0;
    int storage = 0;
    std::vector<int64_t> type_begin;
    std::vector<float> brightness;  // per species
    Mem mem;
    void *attr = nullptr;
    void *meta = nullptr;
    void *emit = nullptr;  // per-particle emission (vector-colour scenes)
    size_t attr_bytes = 0, meta_bytes = 0, emit_bytes = 0;
    SceneDev dev_view{};
};

extern "C" splotch_render_params splotch_default_params(void) {
    splotch_render_params p;
    p.tile = 0;
    p.rfac = 0.75f;
    p.sigma_over_R = 0.5f;
    p.r_min_px = 0.75f;
    p.block_particles = 0;
    p.flags = 0;
    return p;
}

static splotch_status validate_desc(const splotch_scene_desc *d) {
    if (!d) return fail(SPLOTCH_ERR_INVALID_ARG, "desc is NULL");
    if (d->n < 0) return fail(SPLOTCH_ERR_INVALID_ARG, "n < 0");
    if (d->n >= (int64_t)1 << 31) return fail(SPLOTCH_ERR_UNSUPPORTED, "n >= 2^31 particles");
    if (d->n_types < 1 || d->n_types > kMaxTypes)
        return fail(SPLOTCH_ERR_INVALID_ARG, "n_types must be 1..%d", kMaxTypes);
    if (!d->type_begin) return fail(SPLOTCH_ERR_INVALID_ARG, "type_begin is NULL");
    if (d->type_begin[0] != 0 || d->type_begin[d->n_types] != d->n)
        return fail(SPLOTCH_ERR_INVALID_ARG, "type_begin must start at 0 and end at n");
    for (int t = 0; t < d->n_types; ++t)
        if (d->type_begin[t + 1] < d->type_begin[t])
            return fail(SPLOTCH_ERR_INVALID_ARG, "type_begin must be non-decreasing");
    if (d->n > 0 && (!d->x || !d->y || !d->z || !d->h || !d->intensity))
        return fail(SPLOTCH_ERR_INVALID_ARG, "particle array is NULL");
    if (d->storage < 0 || d->storage > 2) return fail(SPLOTCH_ERR_INVALID_ARG, "bad storage");
    if (!d->cmap_rgb || !d->cmap_len || !d->brightness || !d->i_log)
        return fail(SPLOTCH_ERR_INVALID_ARG, "per-type array is NULL");
    if ((d->i_min == nullptr) != (d->i_max == nullptr))
        return fail(SPLOTCH_ERR_INVALID_ARG, "give both i_min and i_max or neither");
    for (int t = 0; t < d->n_types; ++t) {
        if (d->cmap_len[t] < 2 || d->cmap_len[t] > (1 << 20))
            return fail(SPLOTCH_ERR_INVALID_ARG, "colormap %d needs 2..2^20 entries", t);
        if (!d->cmap_rgb[t]) return fail(SPLOTCH_ERR_INVALID_ARG, "colormap %d is NULL", t);
        for (int k = 0; k < 3 * d->cmap_len[t]; ++k)
            if (!std::isfinite(d->cmap_rgb[t][k])) return fail(SPLOTCH_ERR_INVALID_ARG, "colormap %d not finite", t);
        if (!std::isfinite(d->brightness[t])) return fail(SPLOTCH_ERR_INVALID_ARG, "brightness not finite");
        if (d->i_min && !(std::isfinite(d->i_min[t]) && std::isfinite(d->i_max[t])))
            return fail(SPLOTCH_ERR_INVALID_ARG, "intensity range not finite");
    }
    if ((d->allocator.alloc == nullptr) != (d->allocator.free == nullptr))
        return fail(SPLOTCH_ERR_INVALID_ARG, "give both allocator callbacks or neither");
    if (d->col_vector && d->n > 0 && !d->rgb) {
        for (int t = 0; t < d->n_types; ++t)
            if (d->col_vector[t]) return fail(SPLOTCH_ERR_INVALID_ARG, "vector-coloured species %d without rgb", t);
    }
    return SPLOTCH_OK;
}

static float order_key_inv(unsigned k) {
    unsigned b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

// copy_engine: stage page-locked host inputs with asynchronous copies (the copy engine)
// instead of reading them in place with the preparation kernel: slower alone, but the
// copy then overlaps kernels that occupy every SM (the out-of-core render).
static splotch_status create_scene_impl(const splotch_scene_desc *d, splotch_scene **out, bool copy_engine);

extern "C" splotch_status splotch_create_scene(const splotch_scene_desc *d, splotch_scene **out) {
    return create_scene_impl(d, out, false);
}

// Per-particle emission of a scene with vector-coloured species (the scene's attributes
// and colormaps are already on the device): ranges of the vector species' colour
// components (given, or their joint min / max), then k_emission.  Sets sc->emit.
static splotch_status build_emission(const splotch_scene_desc *d, splotch_scene *sc, bool copy_engine) {
    cudaStream_t st = (cudaStream_t)d->stream;
    sc->emit_bytes = align256(sizeof(float4) * (size_t)std::max<int64_t>(1, d->n));
    sc->emit = sc->mem.alloc(sc->emit_bytes, st);
    if (!sc->emit) return fail(SPLOTCH_ERR_OOM, "per-particle emission (%zu bytes)", sc->emit_bytes);
    if (d->n == 0) return SPLOTCH_OK;
    const int nt = d->n_types;
    const size_t fb = sizeof(float) * 3 * (size_t)d->n;
    // the colour field on the device: as given, through its device-visible address when
    // page-locked, else staged
    const float *rgb = d->on_device ? d->rgb : nullptr;
    if (!rgb && !copy_engine) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, d->rgb) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            rgb = (const float *)pa.devicePointer;
        else
            cudaGetLastError();
    }
    Carve sv;
    const size_t o_rgb = rgb ? 0 : sv.take(fb);
    const size_t o_vec = sv.take(sizeof(int) * nt), o_lo = sv.take(sizeof(float) * nt);
    const size_t o_hi = sv.take(sizeof(float) * nt), o_lg = sv.take(sizeof(int) * nt);
    const size_t o_beta = sv.take(sizeof(float) * nt), o_keys = sv.take(sizeof(unsigned) * 2 * nt);
    const size_t o_bad = sv.take(sizeof(int));
    char *stg = (char *)sc->mem.alloc(sv.off, st);
    if (!stg) return fail(SPLOTCH_ERR_OOM, "emission staging");
    if (!rgb) {
        cudaMemcpyAsync(stg + o_rgb, d->rgb, fb, cudaMemcpyHostToDevice, st);
        rgb = (const float *)(stg + o_rgb);
    }
    std::vector<int> vec(nt), lg(d->i_log, d->i_log + nt);
    std::vector<float> lo(nt, 0.0f), hi(nt, 0.0f);
    for (int t = 0; t < nt; ++t) vec[t] = d->col_vector[t] != 0;
    if (d->i_min) {
        for (int t = 0; t < nt; ++t) lo[t] = d->i_min[t], hi[t] = d->i_max[t];
    } else {
        std::vector<unsigned> keys(2 * nt);
        for (int t = 0; t < nt; ++t) keys[2 * t] = 0xFFFFFFFFu, keys[2 * t + 1] = 0u;
        cudaMemcpyAsync(stg + o_keys, keys.data(), sizeof(unsigned) * keys.size(), cudaMemcpyHostToDevice, st);
        for (int t = 0; t < nt; ++t) {
            if (!vec[t]) continue;
            cudaError_t e = launch_minmax(0, rgb, 3 * d->type_begin[t], 3 * d->type_begin[t + 1], d->i_log[t],
                                          (unsigned *)(stg + o_keys) + 2 * t, st);
            if (e != cudaSuccess) {
                sc->mem.release(stg, st);
                return fail(SPLOTCH_ERR_CUDA, "colour range: %s", cudaGetErrorString(e));
            }
        }
        cudaMemcpyAsync(keys.data(), stg + o_keys, sizeof(unsigned) * keys.size(), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        for (int t = 0; t < nt; ++t) {
            lo[t] = keys[2 * t] == 0xFFFFFFFFu ? 0.0f : order_key_inv(keys[2 * t]);
            hi[t] = keys[2 * t + 1] == 0u ? 0.0f : order_key_inv(keys[2 * t + 1]);
        }
    }
    cudaMemcpyAsync(stg + o_vec, vec.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(stg + o_lo, lo.data(), sizeof(float) * nt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(stg + o_hi, hi.data(), sizeof(float) * nt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(stg + o_lg, lg.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(stg + o_beta, d->brightness, sizeof(float) * nt, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(stg + o_bad, 0, sizeof(int), st);
    cudaError_t e = launch_emission(sc->storage, sc->dev_view, rgb, (const int *)(stg + o_vec),
                                    (const float *)(stg + o_lo), (const float *)(stg + o_hi),
                                    (const int *)(stg + o_lg), (const float *)(stg + o_beta), (float4 *)sc->emit,
                                    (int *)(stg + o_bad), st);
    int bad = 0;
    cudaMemcpyAsync(&bad, stg + o_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    sc->mem.release(stg, st);
    if (e != cudaSuccess || se != cudaSuccess)
        return fail(SPLOTCH_ERR_CUDA, "emission: %s", cudaGetErrorString(e != cudaSuccess ? e : se));
    if (bad) return fail(SPLOTCH_ERR_INVALID_ARG, "non-finite colour component");
    sc->dev_view.emit = (const float4 *)sc->emit;
    return SPLOTCH_OK;
}

static splotch_status create_scene_impl(const splotch_scene_desc *d, splotch_scene **out, bool copy_engine) {
    if (!out) return fail(SPLOTCH_ERR_INVALID_ARG, "out is NULL");
    splotch_status s = validate_desc(d);
    if (s != SPLOTCH_OK) return s;
    cudaStream_t st = (cudaStream_t)d->stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));

    splotch_scene *sc = new splotch_scene();
    sc->dev = dev;
    sc->n = d->n;
    sc->n_pad = ((d->n + 7) / 8) * 8 + 8;
    sc->n_types = d->n_types;
    sc->storage = d->storage;
    sc->type_begin.assign(d->type_begin, d->type_begin + d->n_types + 1);
    sc->brightness.assign(d->brightness, d->brightness + d->n_types);
    sc->mem.a = d->allocator;
    sc->mem.dev = dev;

    auto cleanup = [&](splotch_status st_) {
        if (sc->attr) sc->mem.release(sc->attr, st);
        if (sc->meta) sc->mem.release(sc->meta, st);
        if (sc->emit) sc->mem.release(sc->emit, st);
        cudaStreamSynchronize(st);
        delete sc;
        return st_;
    };

    const size_t elem = d->storage == 0 ? 4 : 2;
    const size_t arr = align256((size_t)sc->n_pad * elem);
    sc->attr_bytes = 5 * arr;
    sc->attr = sc->mem.alloc(sc->attr_bytes, st);
    if (!sc->attr) return cleanup(fail(SPLOTCH_ERR_OOM, "scene attributes (%zu bytes)", sc->attr_bytes));

    // colormaps premultiplied by brightness, as float4
    std::vector<int> lut_off(d->n_types), lut_len(d->n_types);
    int total = 0;
    for (int t = 0; t < d->n_types; ++t) {
        lut_off[t] = total;
        lut_len[t] = d->cmap_len[t];
        total += d->cmap_len[t];
    }
    std::vector<float> lut(4 * (size_t)total);
    for (int t = 0; t < d->n_types; ++t)
        for (int k = 0; k < d->cmap_len[t]; ++k) {
            for (int c = 0; c < 3; ++c)
                lut[4 * (lut_off[t] + k) + c] = d->brightness[t] * d->cmap_rgb[t][3 * k + c];
            lut[4 * (lut_off[t] + k) + 3] = 0.0f;
        }
    Carve cv;
    const size_t o_tb = cv.take(sizeof(int64_t) * (d->n_types + 1));
    const size_t o_lut = cv.take(sizeof(float) * lut.size());
    const size_t o_off = cv.take(sizeof(int) * d->n_types);
    const size_t o_len = cv.take(sizeof(int) * d->n_types);
    sc->meta_bytes = cv.off;
    sc->meta = sc->mem.alloc(sc->meta_bytes, st);
    if (!sc->meta) return cleanup(fail(SPLOTCH_ERR_OOM, "scene metadata"));
    char *mb = (char *)sc->meta;
    cudaMemcpyAsync(mb + o_tb, d->type_begin, sizeof(int64_t) * (d->n_types + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(mb + o_lut, lut.data(), sizeof(float) * lut.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(mb + o_off, lut_off.data(), sizeof(int) * d->n_types, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(mb + o_len, lut_len.data(), sizeof(int) * d->n_types, cudaMemcpyHostToDevice, st);

    char *ab = (char *)sc->attr;
    // the preparation kernel writes [0, n) of every array; zero the padding behind it
    for (int k = 0; k < 5; ++k)
        if (cudaMemsetAsync(ab + k * arr + (size_t)d->n * elem, 0, arr - (size_t)d->n * elem, st) != cudaSuccess)
            return cleanup(fail(SPLOTCH_ERR_CUDA, "memset scene"));

    if (d->n > 0) {
        // Host inputs in page-locked memory are read by the preparation kernel in place
        // (through their device-visible address: no staging copy); pageable host inputs
        // are staged on the device first.
        const float *src[5] = {d->x, d->y, d->z, d->h, d->intensity};
        const float *in[5];
        bool copy_in = !d->on_device;
        if (copy_in && !copy_engine) {
            bool pinned = true;
            for (int k = 0; k < 5 && pinned; ++k) {
                cudaPointerAttributes pa{};
                if (cudaPointerGetAttributes(&pa, src[k]) != cudaSuccess) {
                    cudaGetLastError();
                    pinned = false;
                } else if (pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
                    pinned = false;
                } else {
                    in[k] = (const float *)pa.devicePointer;
                }
            }
            copy_in = !pinned;
        }
        // staging: FP32 inputs on the device (pageable host inputs only), per-type range,
        // validity flag
        Carve sv;
        const size_t f = sizeof(float) * (size_t)d->n;
        size_t o_in[5] = {0, 0, 0, 0, 0};
        if (copy_in)
            for (int k = 0; k < 5; ++k) o_in[k] = sv.take(f);
        const size_t o_lo = sv.take(sizeof(float) * d->n_types);
        const size_t o_hi = sv.take(sizeof(float) * d->n_types);
        const size_t o_lg = sv.take(sizeof(int) * d->n_types);
        const size_t o_keys = sv.take(sizeof(unsigned) * 2 * d->n_types);
        const size_t o_bad = sv.take(sizeof(int));
        char *stg = (char *)sc->mem.alloc(sv.off, st);
        if (!stg) return cleanup(fail(SPLOTCH_ERR_OOM, "scene staging"));
        for (int k = 0; k < 5; ++k) {
            if (copy_in) {
                cudaMemcpyAsync(stg + o_in[k], src[k], f, cudaMemcpyHostToDevice, st);
                in[k] = (const float *)(stg + o_in[k]);
            } else if (d->on_device) {
                in[k] = src[k];
            }
        }
        std::vector<int> lg(d->i_log, d->i_log + d->n_types);
        cudaMemcpyAsync(stg + o_lg, lg.data(), sizeof(int) * d->n_types, cudaMemcpyHostToDevice, st);
        std::vector<float> lo(d->n_types), hi(d->n_types);
        if (d->i_min) {
            for (int t = 0; t < d->n_types; ++t) {
                lo[t] = d->i_min[t];
                hi[t] = d->i_max[t];
            }
        } else {
            std::vector<unsigned> keys(2 * d->n_types);
            for (int t = 0; t < d->n_types; ++t) {
                keys[2 * t] = 0xFFFFFFFFu;
                keys[2 * t + 1] = 0u;
            }
            cudaMemcpyAsync(stg + o_keys, keys.data(), sizeof(unsigned) * keys.size(), cudaMemcpyHostToDevice, st);
            for (int t = 0; t < d->n_types; ++t) {
                cudaError_t e = launch_minmax(0, in[4], d->type_begin[t], d->type_begin[t + 1], d->i_log[t],
                                              (unsigned *)(stg + o_keys) + 2 * t, st);
                if (e != cudaSuccess) {
                    sc->mem.release(stg, st);
                    return cleanup(fail(SPLOTCH_ERR_CUDA, "minmax: %s", cudaGetErrorString(e)));
                }
            }
            cudaMemcpyAsync(keys.data(), stg + o_keys, sizeof(unsigned) * keys.size(), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            for (int t = 0; t < d->n_types; ++t) {
                lo[t] = keys[2 * t] == 0xFFFFFFFFu ? 0.0f : order_key_inv(keys[2 * t]);
                hi[t] = keys[2 * t + 1] == 0u ? 0.0f : order_key_inv(keys[2 * t + 1]);
            }
        }
        cudaMemcpyAsync(stg + o_lo, lo.data(), sizeof(float) * d->n_types, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(stg + o_hi, hi.data(), sizeof(float) * d->n_types, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(stg + o_bad, 0, sizeof(int), st);
        cudaError_t e = launch_prepare(in[0], in[1], in[2], in[3], in[4], d->n, d->n_types,
                                       (const int64_t *)(mb + o_tb), (const float *)(stg + o_lo),
                                       (const float *)(stg + o_hi), (const int *)(stg + o_lg), d->storage,
                                       ab, ab + arr, ab + 2 * arr, ab + 3 * arr, ab + 4 * arr,
                                       (int *)(stg + o_bad), st);
        int bad = 0;
        cudaMemcpyAsync(&bad, stg + o_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaError_t se = cudaStreamSynchronize(st);
        sc->mem.release(stg, st);
        if (e != cudaSuccess || se != cudaSuccess)
            return cleanup(fail(SPLOTCH_ERR_CUDA, "prepare: %s", cudaGetErrorString(e != cudaSuccess ? e : se)));
        if (bad) return cleanup(fail(SPLOTCH_ERR_INVALID_ARG, "non-finite attribute or h <= 0"));
    }
    cudaError_t se = cudaStreamSynchronize(st);
    if (se != cudaSuccess) return cleanup(fail(SPLOTCH_ERR_CUDA, "create: %s", cudaGetErrorString(se)));

    SceneDev &v = sc->dev_view;
    v.emit = nullptr;
    v.x = ab;
    v.y = ab + arr;
    v.z = ab + 2 * arr;
    v.h = ab + 3 * arr;
    v.it = ab + 4 * arr;
    v.n = sc->n;
    v.n_types = sc->n_types;
    v.type_begin = (const int64_t *)(mb + o_tb);
    v.lut = (const float4 *)(mb + o_lut);
    v.lut_off = (const int *)(mb + o_off);
    v.lut_len = (const int *)(mb + o_len);
    bool any_vec = false;
    for (int t = 0; d->col_vector && t < d->n_types; ++t) any_vec |= d->col_vector[t] != 0;
    if (any_vec) {
        s = build_emission(d, sc, copy_engine);
        if (s != SPLOTCH_OK) return cleanup(s);
    }
    *out = sc;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_destroy(splotch_scene *sc) {
    if (!sc) return SPLOTCH_OK;
    sc->mem.release(sc->attr, 0);
    sc->mem.release(sc->meta, 0);
    sc->mem.release(sc->emit, 0);
    cudaStreamSynchronize(0);
    delete sc;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_scene_info(const splotch_scene *sc, int64_t *n, int32_t *n_types,
                                             int32_t *storage, int64_t *device_bytes) {
    if (!sc) return fail(SPLOTCH_ERR_INVALID_ARG, "scene is NULL");
    if (n) *n = sc->n;
    if (n_types) *n_types = sc->n_types;
    if (storage) *storage = sc->storage;
    if (device_bytes) *device_bytes = (int64_t)(sc->attr_bytes + sc->meta_bytes + sc->emit_bytes);
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// camera (FP64, each operation rounded once, then each entry rounded to FP32)

static double dot3(const double *a, const double *b) {
    double t = a[0] * b[0];
    t = t + a[1] * b[1];
    t = t + a[2] * b[2];
    return t;
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static splotch_status compose_camera(const splotch_camera *c, float m[12], float p[5]) {
    if (!c) return fail(SPLOTCH_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "image size < 1");
    if (!(c->fov_deg > 0.0 && c->fov_deg < 180.0)) return fail(SPLOTCH_ERR_INVALID_ARG, "fov outside (0, 180)");
    if (!(c->z_near > 0.0)) return fail(SPLOTCH_ERR_INVALID_ARG, "z_near <= 0");
    const bool has_far = c->z_far > 0.0 && std::isfinite(c->z_far);
    if (has_far && !(c->z_far > c->z_near)) return fail(SPLOTCH_ERR_INVALID_ARG, "z_far <= z_near");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(c->eye[k]) || !std::isfinite(c->lookat[k]) || !std::isfinite(c->up[k]))
            return fail(SPLOTCH_ERR_INVALID_ARG, "camera not finite");
    const double d[3] = {c->lookat[0] - c->eye[0], c->lookat[1] - c->eye[1], c->lookat[2] - c->eye[2]};
    const double nd = std::sqrt(dot3(d, d));
    if (!(nd > 0.0)) return fail(SPLOTCH_ERR_INVALID_ARG, "eye == lookat");
    const double f[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
    double s0[3];
    cross3(f, c->up, s0);
    const double ns = std::sqrt(dot3(s0, s0));
    const double nu = std::sqrt(dot3(c->up, c->up));
    if (!(ns > 1e-9 * nu)) return fail(SPLOTCH_ERR_INVALID_ARG, "up vector parallel to the view direction");
    const double s[3] = {s0[0] / ns, s0[1] / ns, s0[2] / ns};
    double u[3];
    cross3(s, f, u);
    const double *rows[3] = {s, u, f};
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) m[4 * r + k] = (float)rows[r][k];
        m[4 * r + 3] = (float)(-dot3(rows[r], c->eye));
    }
    const double F = (0.5 * (double)c->height) / std::tan(c->fov_deg * (M_PI / 360.0));
    p[0] = (float)F;
    p[1] = 0.5f * (float)c->width;
    p[2] = 0.5f * (float)c->height;
    p[3] = (float)c->z_near;
    p[4] = has_far ? (float)c->z_far : INFINITY;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_camera_params(const splotch_camera *cam, float m[12], float p[5]) {
    if (!m || !p) return fail(SPLOTCH_ERR_INVALID_ARG, "output is NULL");
    return compose_camera(cam, m, p);
}

// Output mode of the splat kernels: 0 final transform, 1 write a, 2 add a.
static int out_mode(int flags) {
    return (flags & SPLOTCH_OUT_ADD) ? 2 : ((flags & SPLOTCH_OUT_ACCUM) ? 1 : 0);
}

static splotch_status check_params(const splotch_render_params *pr) {
    if (!(pr->rfac > 0.0f) || !std::isfinite(pr->rfac)) return fail(SPLOTCH_ERR_INVALID_ARG, "rfac <= 0");
    if (!(pr->sigma_over_R > 0.0f) || !std::isfinite(pr->sigma_over_R))
        return fail(SPLOTCH_ERR_INVALID_ARG, "sigma_over_R <= 0");
    if (!(pr->r_min_px >= 0.0f) || !std::isfinite(pr->r_min_px)) return fail(SPLOTCH_ERR_INVALID_ARG, "r_min_px < 0");
    if (pr->tile < 0 || pr->tile > kMaxTile) return fail(SPLOTCH_ERR_INVALID_ARG, "tile outside 0..%d", kMaxTile);
    if (pr->block_particles < 0) return fail(SPLOTCH_ERR_INVALID_ARG, "block_particles < 0");
    return SPLOTCH_OK;
}

static int64_t n_tiles_for(int W, int H, int T) {
    return (int64_t)((W + T - 1) / T) * ((H + T - 1) / T);
}

static splotch_status choose_tile(int W, int H, int requested, int *T) {
    if (requested > 0) {
        if (n_tiles_for(W, H, requested) > kMaxTiles)
            return fail(SPLOTCH_ERR_UNSUPPORTED, "tile %d gives more than %d tiles for %dx%d", requested,
                        kMaxTiles, W, H);
        *T = requested;
        return SPLOTCH_OK;
    }
    for (int t = 16; t <= kMaxTile; t += 8)
        if (n_tiles_for(W, H, t) <= kMaxTiles) {
            *T = t;
            return SPLOTCH_OK;
        }
    return fail(SPLOTCH_ERR_UNSUPPORTED, "image %dx%d needs more than %d tiles of %d px", W, H, kMaxTiles, kMaxTile);
}

static splotch_status make_view(const splotch_camera *c, const splotch_render_params &pr, int T, ViewParams &v) {
    float m[12], p[5];
    splotch_status s = compose_camera(c, m, p);
    if (s != SPLOTCH_OK) return s;
    memcpy(v.m, m, sizeof(m));
    v.F = p[0];
    v.cx = p[1];
    v.cy = p[2];
    v.zn = p[3];
    v.zf = p[4];
    v.rfac = pr.rfac;
    v.rmin = pr.r_min_px;
    v.kexp = -kLog2e / (pr.sigma_over_R * pr.sigma_over_R);
    v.hd = 0.70710677f * (float)T;
    v.W = c->width;
    v.H = c->height;
    v.T = T;
    v.ntx = (c->width + T - 1) / T;
    v.nty = (c->height + T - 1) / T;
    v.n_tiles = v.ntx * v.nty;
    v.fastdiv = (T > 1 && c->width <= 65536 && c->height <= 65536) ? 1 : 0;
    v.tmagic = T > 1 ? (uint32_t)((((uint64_t)1) << 32) / (uint64_t)T + 1) : 0u;
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// frame workspace

struct FrameHost {
    int V = 0, G = 1, T = 32, n_tiles = 0, n_chunks = 1;
    int64_t chunk = 0;
    int storage = 0;
    // fixed part
    size_t o_views, o_counts, o_rel, o_offsets, o_item, o_split, o_sizes, o_status, o_queue, fixed_bytes;
    // variable part (capacities)
    int64_t pair_cap = 0;
    int item_cap = 0, split_cap = 0;
    bool pids = false;
    bool order = false;  // the splat takes its work items largest first (k_item_order)
    size_t o_lists, o_pids, o_scratch, o_tickets, o_order = 0, var_bytes;
};

static const int64_t kRelBudget = 256ll << 20;
static const int kChunkPerEntry = 8;  // particles per histogram entry in a binning chunk

static void layout_fixed(FrameHost &fh, const splotch_scene *sc, int V, int n_tiles, int T,
                         int block_particles = 0, int64_t rel_budget = kRelBudget) {
    fh.V = V;
    fh.T = T;
    fh.n_tiles = n_tiles;
    fh.storage = sc->storage;
    fh.G = std::max(1, std::min({V, kMaxGroup, kMaxTiles / std::max(1, n_tiles)}));
    const int n_sm = sm_count(sc->dev);
    const int vec = sc->storage == 0 ? 4 : 8;
    const int64_t unit = (int64_t)kThreads * vec;
    const int64_t n_units = std::max<int64_t>(1, (sc->n + unit - 1) / unit);
    const int groups = (V + fh.G - 1) / fh.G;
    // Chunks of the binning kernels: whole waves over all view groups, as many as four where
    // every chunk keeps at least kChunkPerEntry particles per histogram entry (its fixed cost
    // is clearing and writing one count per tile), never fewer than two.  With two waves the
    // chunks' unequal costs (a gas particle makes about twice the records of a star) left the
    // last wave's SMs idle for about a sixth of the scatter; a chunk count just above a whole
    // number of waves would add a wave for a few CTAs.
    const int occ = bin_ctas_per_sm(sc->storage, sizeof(int) * (size_t)fh.G * n_tiles);
    const int64_t min_chunk = (int64_t)kChunkPerEntry * fh.G * n_tiles;
    const int64_t max_by_size = std::max<int64_t>(1, sc->n / std::max<int64_t>(1, min_chunk));
    int64_t target = std::max<int64_t>(1, (2ll * n_sm * occ + groups - 1) / groups);
    for (int64_t w = 3; w <= 4; ++w) {
        const int64_t t = std::max<int64_t>(1, (w * n_sm * occ + groups - 1) / groups);
        if (t <= max_by_size) target = t;
    }
    target = std::min(target, n_units);
    const int64_t max_chunks = std::max<int64_t>(1, rel_budget / (4ll * V * n_tiles));
    int64_t nch = std::min(target, max_chunks);
    if (block_particles > 0) nch = std::min(max_chunks, std::max<int64_t>(1, (sc->n + block_particles - 1) / block_particles));
    const int64_t upc = (n_units + nch - 1) / nch;
    fh.chunk = upc * unit;
    fh.n_chunks = (int)std::max<int64_t>(1, (sc->n + fh.chunk - 1) / fh.chunk);
    const int64_t N = (int64_t)V * n_tiles;
    Carve cv;
    fh.o_views = cv.take(sizeof(ViewParams) * V);
    fh.o_counts = cv.take(sizeof(int) * N);
    fh.o_rel = cv.take(sizeof(int) * N * fh.n_chunks);
    fh.o_offsets = cv.take(sizeof(int64_t) * (N + 1));
    fh.o_item = cv.take(sizeof(int) * (N + 1));
    fh.o_split = cv.take(sizeof(int) * N);
    fh.o_sizes = cv.take(sizeof(int64_t) * 8);
    fh.o_status = cv.take(sizeof(int) * 4);
    fh.o_queue = cv.take(sizeof(int) * 4);
    fh.fixed_bytes = cv.off;
}

// Exact accumulators of one split tile: 3 channels x T x T pixels, 16 bytes each.
static size_t split_scratch_bytes(int T) { return sizeof(unsigned long long) * 2 * 3 * (size_t)T * T; }

// order: room for the splat's item order (one int per work item; the fixed-array render
// takes its items in tile order).
static void layout_var(FrameHost &fh, int64_t pairs, int items, int splits, bool pids, bool order = true) {
    fh.pair_cap = pairs;
    fh.item_cap = items;
    fh.split_cap = splits;
    fh.pids = pids;
    fh.order = order;
    Carve cv;
    fh.o_lists = cv.take(sizeof(float4) * std::max<int64_t>(1, pairs));
    fh.o_pids = pids ? cv.take(sizeof(int) * std::max<int64_t>(1, pairs)) : 0;
    fh.o_scratch = cv.take(split_scratch_bytes(fh.T) * std::max(1, splits));
    fh.o_tickets = cv.take(sizeof(int) * std::max(1, splits));
    fh.o_order = order ? cv.take(sizeof(int) * (size_t)std::max(1, items)) : 0;
    fh.var_bytes = cv.off;
}

static FrameDev frame_dev(const FrameHost &fh, char *fixed, char *var) {
    FrameDev fr{};
    fr.views = (const ViewParams *)(fixed + fh.o_views);
    fr.V = fh.V;
    fr.G = fh.G;
    fr.n_tiles = fh.n_tiles;
    fr.T = fh.T;
    fr.chunk = fh.chunk;
    fr.n_chunks = fh.n_chunks;
    fr.counts = (int *)(fixed + fh.o_counts);
    fr.rel = (int *)(fixed + fh.o_rel);
    fr.offsets = (int64_t *)(fixed + fh.o_offsets);
    fr.item_off = (int *)(fixed + fh.o_item);
    fr.split_slot = (int *)(fixed + fh.o_split);
    fr.sizes = (int64_t *)(fixed + fh.o_sizes);
    fr.status = (int *)(fixed + fh.o_status);
    if (var) {
        fr.lists = (float4 *)(var + fh.o_lists);
        fr.pids = fh.pids ? (int *)(var + fh.o_pids) : nullptr;
        fr.scratch = (unsigned long long *)(var + fh.o_scratch);
        fr.tickets = (int *)(var + fh.o_tickets);
        fr.order = fh.order ? (int *)(var + fh.o_order) : nullptr;
    }
    fr.pair_cap = var ? fh.pair_cap : INT64_MAX;
    fr.item_cap = var ? fh.item_cap : INT32_MAX;
    fr.split_cap = var ? fh.split_cap : INT32_MAX;
    return fr;
}

// items: work items of the scan (tile-list slices); the splat renders each as split^2
// squares, one worker each
static int splat_grid(int dev, int T, int items) {
    const int bps = std::max(1, splat_blocks_per_sm(T));
    const int per_cta = std::max(1, splat_workers_per_sm(T) / bps);
    const int g = sm_count(dev) * bps;
    const int64_t squares = (int64_t)std::max(1, items) * splat_split(T) * splat_split(T);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (squares + per_cta - 1) / per_cta));
}

static int target_items(int dev, int T) {
    const int s = splat_split(T);
    return std::max(1, sm_count(dev) * std::max(1, splat_workers_per_sm(T)) * 4 / (s * s));
}
static const int kMinItemPairs = 2048;

struct RenderSetup {
    int W = 0, H = 0, T = 0, V = 0;
    std::vector<ViewParams> views;
    splotch_render_params pr{};
};

static splotch_status setup_views(const splotch_camera *cams, int n_views, const splotch_render_params *params,
                                  RenderSetup &rs) {
    if (!cams) return fail(SPLOTCH_ERR_INVALID_ARG, "cams is NULL");
    if (n_views < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "n_views < 1");
    rs.pr = params ? *params : splotch_default_params();
    splotch_status s = check_params(&rs.pr);
    if (s != SPLOTCH_OK) return s;
    rs.W = cams[0].width;
    rs.H = cams[0].height;
    for (int v = 0; v < n_views; ++v)
        if (cams[v].width != rs.W || cams[v].height != rs.H)
            return fail(SPLOTCH_ERR_INVALID_ARG, "all views must share the image size");
    if (rs.W < 1 || rs.H < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "image size < 1");
    if ((int64_t)rs.W * rs.H > (int64_t)1 << 30) return fail(SPLOTCH_ERR_UNSUPPORTED, "image larger than 2^30 px");
    s = choose_tile(rs.W, rs.H, rs.pr.tile, &rs.T);
    if (s != SPLOTCH_OK) return s;
    rs.V = n_views;
    rs.views.resize(n_views);
    for (int v = 0; v < n_views; ++v) {
        s = make_view(&cams[v], rs.pr, rs.T, rs.views[v]);
        if (s != SPLOTCH_OK) return s;
    }
    return SPLOTCH_OK;
}

// Count + scan for all views and read the sizes back (blocking).
static splotch_status count_and_size(splotch_scene *sc, const RenderSetup &rs, FrameHost &fh, char *fixed,
                                     cudaStream_t st, int64_t sizes[8], cudaEvent_t *ev = nullptr,
                                     int scan_target = 0) {
    FrameDev fr = frame_dev(fh, fixed, nullptr);
    CUDA_TRY(cudaMemcpyAsync(fixed + fh.o_views, rs.views.data(), sizeof(ViewParams) * rs.V,
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(fixed + fh.o_counts, 0, sizeof(int) * (size_t)rs.V * fh.n_tiles, st));
    CUDA_TRY(cudaMemsetAsync(fixed + fh.o_status, 0, sizeof(int) * 4, st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[0], st));
    CUDA_TRY(launch_count(sc->storage, sc->dev_view, fr, st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[1], st));
    CUDA_TRY(launch_scan(fr, scan_target > 0 ? scan_target : target_items(sc->dev, fh.T), kMinItemPairs, st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[2], st));
    int64_t *box = host_box();
    if (!box) return fail(SPLOTCH_ERR_OOM, "pinned host buffer");
    CUDA_TRY(cudaMemcpyAsync(box, fixed + fh.o_sizes, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(sizes, box, sizeof(int64_t) * 8);
    return SPLOTCH_OK;
}

// Enqueue scatter + splat for a sized frame.
static splotch_status scatter_and_splat(splotch_scene *sc, FrameHost &fh, char *fixed, char *var, float *out,
                                        int out_accum, bool stable, int items, cudaStream_t st,
                                        cudaEvent_t *ev = nullptr) {
    FrameDev fr = frame_dev(fh, fixed, var);
    CUDA_TRY(cudaMemsetAsync(fixed + fh.o_queue, 0, sizeof(int) * 4, st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[3], st));
    CUDA_TRY(launch_scatter(sc->storage, sc->dev_view, fr, stable, st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[4], st));
    CUDA_TRY(launch_splat(sc->dev_view, fr, (int *)(fixed + fh.o_queue), out, out_accum,
                          splat_grid(sc->dev, fh.T, items), st));
    if (ev) CUDA_TRY(cudaEventRecord(ev[5], st));
    return SPLOTCH_OK;
}


static splotch_status render_frame(splotch_scene *sc, const RenderSetup &rs, float *out, cudaStream_t st,
                                   bool sync, bool want_pids, int32_t *dbg_counts, int64_t *dbg_offsets,
                                   int32_t *dbg_members, int64_t dbg_cap, int64_t *dbg_total) {
    FrameHost fh;
    layout_fixed(fh, sc, rs.V, rs.views[0].n_tiles, rs.T, rs.pr.block_particles);
    const bool timed = (rs.pr.flags & SPLOTCH_TIMING) != 0 && !dbg_members;
    cudaEvent_t *ev = nullptr;
    if (timed) {
        if (!g_timing.init()) return fail(SPLOTCH_ERR_CUDA, "timing events");
        ev = g_timing.ev;
        g_timing.have = false;
        sync = true;
    }
    char *fixed = (char *)sc->mem.alloc(fh.fixed_bytes, st);
    if (!fixed) return fail(SPLOTCH_ERR_OOM, "frame workspace (%zu bytes)", fh.fixed_bytes);
    int64_t sizes[8];
    splotch_status s = count_and_size(sc, rs, fh, fixed, st, sizes, ev);
    if (s != SPLOTCH_OK) {
        sc->mem.release(fixed, st);
        return s;
    }
    const int64_t P = sizes[kSizePairs];
    const int items = (int)sizes[kSizeItems], splits = (int)sizes[kSizeSplits];
    if (dbg_total) *dbg_total = P;
    if (dbg_members && P > dbg_cap) {
        sc->mem.release(fixed, st);
        return fail(SPLOTCH_ERR_CAPACITY, "member capacity %lld < %lld pairs", (long long)dbg_cap, (long long)P);
    }
    layout_var(fh, P, items, splits, want_pids);
    char *var = (char *)sc->mem.alloc(fh.var_bytes, st);
    if (!var) {
        sc->mem.release(fixed, st);
        return fail(SPLOTCH_ERR_OOM, "tile lists (%zu bytes for %lld pairs)", fh.var_bytes, (long long)P);
    }
    s = SPLOTCH_OK;
    do {
        if (cudaMemsetAsync(var + fh.o_scratch, 0, fh.o_tickets - fh.o_scratch + sizeof(int) * std::max(1, splits),
                            st) != cudaSuccess) {
            s = fail(SPLOTCH_ERR_CUDA, "memset scratch");
            break;
        }
        if (dbg_members) {
            FrameDev fr = frame_dev(fh, fixed, var);
            cudaError_t e = launch_scatter(sc->storage, sc->dev_view, fr, true, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dbg_counts, fixed + fh.o_counts, sizeof(int) * fh.n_tiles, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dbg_offsets, fixed + fh.o_offsets, sizeof(int64_t) * (fh.n_tiles + 1),
                                    cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && P > 0)
                e = cudaMemcpyAsync(dbg_members, var + fh.o_pids, sizeof(int) * P, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = fail(SPLOTCH_ERR_CUDA, "debug bins: %s", cudaGetErrorString(e));
            break;
        }
        s = scatter_and_splat(sc, fh, fixed, var, out, out_mode(rs.pr.flags), (rs.pr.flags & SPLOTCH_STABLE) != 0,
                              items, st, ev);
        if (s != SPLOTCH_OK) break;
        if (sync) {
            int64_t *box = host_box();
            if (!box) {
                s = fail(SPLOTCH_ERR_OOM, "pinned host buffer");
                break;
            }
            cudaError_t e = cudaMemcpyAsync(box, fixed + fh.o_status, sizeof(int) * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                s = fail(SPLOTCH_ERR_CUDA, "render: %s", cudaGetErrorString(e));
                break;
            }
            const int *stat = (const int *)box;
            if (stat[kStatTimeout]) s = fail(SPLOTCH_ERR_TIMEOUT, "splat stage wait timed out");
            if (timed && s == SPLOTCH_OK) {
                float t[4] = {0, 0, 0, 0};
                cudaEventElapsedTime(&t[0], ev[0], ev[1]);
                cudaEventElapsedTime(&t[1], ev[1], ev[2]);
                cudaEventElapsedTime(&t[2], ev[3], ev[4]);
                cudaEventElapsedTime(&t[3], ev[4], ev[5]);
                for (int k = 0; k < 4; ++k) g_timing.ms[k] = t[k];
                g_timing.counts[0] = P;
                g_timing.counts[1] = items;
                g_timing.counts[2] = splits;
                g_timing.have = true;
            }
        }
    } while (0);
    sc->mem.release(var, st);
    sc->mem.release(fixed, st);
    return s;
}

extern "C" splotch_status splotch_render(splotch_scene *sc, const splotch_camera *cams, int32_t n_views,
                                         const splotch_render_params *params, float *out, void *stream) {
    if (!sc) return fail(SPLOTCH_ERR_INVALID_ARG, "scene is NULL");
    if (!out) return fail(SPLOTCH_ERR_INVALID_ARG, "out is NULL");
    RenderSetup rs;
    splotch_status s = setup_views(cams, n_views, params, rs);
    if (s != SPLOTCH_OK) return s;
    return render_frame(sc, rs, out, (cudaStream_t)stream, (rs.pr.flags & SPLOTCH_SYNC) != 0, false, nullptr,
                        nullptr, nullptr, 0, nullptr);
}

extern "C" splotch_status splotch_debug_raster(splotch_scene *sc, const splotch_camera *cam,
                                               const splotch_render_params *params, float *out8, void *stream) {
    if (!sc || !out8) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    RenderSetup rs;
    splotch_status s = setup_views(cam, 1, params, rs);
    if (s != SPLOTCH_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    void *vp = sc->mem.alloc(sizeof(ViewParams), st);
    if (!vp) return fail(SPLOTCH_ERR_OOM, "view params");
    cudaError_t e = cudaMemcpyAsync(vp, rs.views.data(), sizeof(ViewParams), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_debug_raster(sc->storage, sc->dev_view, (const ViewParams *)vp, out8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    sc->mem.release(vp, st);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "debug raster: %s", cudaGetErrorString(e));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_debug_bins(splotch_scene *sc, const splotch_camera *cam,
                                             const splotch_render_params *params, int32_t *counts, int64_t *offsets,
                                             int32_t *members, int64_t capacity, int64_t *total, void *stream) {
    if (!sc || !counts || !offsets || !members || !total) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    RenderSetup rs;
    splotch_status s = setup_views(cam, 1, params, rs);
    if (s != SPLOTCH_OK) return s;
    return render_frame(sc, rs, nullptr, (cudaStream_t)stream, true, true, counts, offsets, members, capacity, total);
}

extern "C" int64_t splotch_workspace_bytes(const splotch_scene *sc, int32_t width, int32_t height, int32_t tile,
                                           int64_t pairs) {
    if (!sc || width < 1 || height < 1) return -1;
    int T = 0;
    if (choose_tile(width, height, tile, &T) != SPLOTCH_OK) return -1;
    FrameHost fh;
    layout_fixed(fh, sc, 1, (int)n_tiles_for(width, height, T), T);
    const int64_t nt = n_tiles_for(width, height, T);
    const int64_t splits = std::min<int64_t>(nt, pairs / kMinItemPairs + 1);
    layout_var(fh, pairs, (int)(nt + pairs / kMinItemPairs + 1), (int)splits, false);
    return (int64_t)(fh.fixed_bytes + fh.var_bytes);
}

// -----------------------------------------------------------------------------------------
// two-phase frame: the count pass first, with the exact workspace of the rest reported,
// so that a caller sharing the device (a request server) can reserve it before the
// library allocates it

struct splotch_frame {
    splotch_scene *sc = nullptr;
    RenderSetup rs;
    FrameHost fh;
    char *fixed = nullptr, *var = nullptr;
    cudaStream_t st = nullptr;
    int64_t sizes[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

extern "C" int64_t splotch_frame_fixed_bytes(const splotch_scene *sc, const splotch_camera *cam,
                                             const splotch_render_params *params) {
    if (!sc || !cam) return -1;
    RenderSetup rs;
    if (setup_views(cam, 1, params, rs) != SPLOTCH_OK) return -1;
    FrameHost fh;
    layout_fixed(fh, sc, 1, rs.views[0].n_tiles, rs.T, rs.pr.block_particles);
    return (int64_t)fh.fixed_bytes;
}

extern "C" splotch_status splotch_frame_prepare(splotch_scene *sc, const splotch_camera *cam,
                                                const splotch_render_params *params, void *stream,
                                                splotch_frame **out, int64_t *fixed_bytes, int64_t *var_bytes,
                                                int64_t *pairs) {
    if (!sc || !cam || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    splotch_frame *f = new splotch_frame();
    f->sc = sc;
    f->st = (cudaStream_t)stream;
    splotch_status s = setup_views(cam, 1, params, f->rs);
    if (s != SPLOTCH_OK) {
        delete f;
        return s;
    }
    layout_fixed(f->fh, sc, 1, f->rs.views[0].n_tiles, f->rs.T, f->rs.pr.block_particles);
    f->fixed = (char *)sc->mem.alloc(f->fh.fixed_bytes, f->st);
    if (!f->fixed) {
        delete f;
        return fail(SPLOTCH_ERR_OOM, "frame workspace (%zu bytes)", f->fh.fixed_bytes);
    }
    s = count_and_size(sc, f->rs, f->fh, f->fixed, f->st, f->sizes);
    if (s != SPLOTCH_OK) {
        splotch_frame_destroy(f);
        return s;
    }
    layout_var(f->fh, f->sizes[kSizePairs], (int)f->sizes[kSizeItems], (int)f->sizes[kSizeSplits], false);
    if (fixed_bytes) *fixed_bytes = (int64_t)f->fh.fixed_bytes;
    if (var_bytes) *var_bytes = (int64_t)f->fh.var_bytes;
    if (pairs) *pairs = f->sizes[kSizePairs];
    *out = f;
    return SPLOTCH_OK;
}

// Order stream `st` after everything enqueued so far on the frame's stream, and make `st`
// the frame's stream (its workspace is released in that order).
static splotch_status frame_follow(splotch_frame *f, cudaStream_t st) {
    if (st == f->st) return SPLOTCH_OK;
    cudaEvent_t ev = nullptr;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, f->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "stream order: %s", cudaGetErrorString(e));
    f->st = st;
    return SPLOTCH_OK;
}

// The list phase of a prepared frame: its exact list workspace, then the scatter.
static splotch_status frame_scatter(splotch_frame *f, cudaStream_t st) {
    if (f->var) return fail(SPLOTCH_ERR_INVALID_ARG, "frame already rendered");
    splotch_status s = frame_follow(f, st);
    if (s != SPLOTCH_OK) return s;
    f->var = (char *)f->sc->mem.alloc(f->fh.var_bytes, st);
    if (!f->var) return fail(SPLOTCH_ERR_OOM, "tile lists (%zu bytes)", f->fh.var_bytes);
    CUDA_TRY(cudaMemsetAsync(f->var + f->fh.o_scratch, 0, f->fh.var_bytes - f->fh.o_scratch, st));
    CUDA_TRY(cudaMemsetAsync(f->fixed + f->fh.o_queue, 0, sizeof(int) * 4, st));
    CUDA_TRY(launch_scatter(f->sc->storage, f->sc->dev_view, frame_dev(f->fh, f->fixed, f->var),
                            (f->rs.pr.flags & SPLOTCH_STABLE) != 0, st));
    return SPLOTCH_OK;
}

// The splat of a frame whose lists are built, into `out`.
static splotch_status frame_splat(splotch_frame *f, float *out, cudaStream_t st) {
    splotch_status s = frame_follow(f, st);
    if (s != SPLOTCH_OK) return s;
    CUDA_TRY(launch_splat(f->sc->dev_view, frame_dev(f->fh, f->fixed, f->var), (int *)(f->fixed + f->fh.o_queue),
                          out, out_mode(f->rs.pr.flags), splat_grid(f->sc->dev, f->fh.T, (int)f->sizes[kSizeItems]),
                          st));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_frame_render(splotch_frame *f, float *out, void *stream) {
    if (!f || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    splotch_status s = frame_scatter(f, st);
    if (s == SPLOTCH_OK) s = frame_splat(f, out, st);
    if (s != SPLOTCH_OK || !(f->rs.pr.flags & SPLOTCH_SYNC)) return s;
    int64_t *box = host_box();
    if (!box) return fail(SPLOTCH_ERR_OOM, "pinned host buffer");
    cudaError_t e = cudaMemcpyAsync(box, f->fixed + f->fh.o_status, sizeof(int) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    if (((const int *)box)[kStatTimeout]) return fail(SPLOTCH_ERR_TIMEOUT, "splat stage wait timed out");
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_frame_destroy(splotch_frame *f) {
    if (!f) return SPLOTCH_OK;
    if (f->var) f->sc->mem.release(f->var, f->st);
    if (f->fixed) f->sc->mem.release(f->fixed, f->st);
    delete f;
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// plan: pre-sized multi-view frame, launchable without host synchronisation

struct splotch_plan {
    splotch_scene *sc = nullptr;
    RenderSetup rs;
    FrameHost fh;
    char *fixed = nullptr, *var = nullptr;
    int grid = 1;
    int64_t *box = nullptr;  // pinned: sizes[8] then status[4] (as ints)
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    float *exec_out = nullptr;
    float *vscale = nullptr;  // device [V * n_types] emission scale per view and species
    // per-view colormaps: device [2 * V * n_types] (offsets, then lengths) into vlut, which
    // is the scene's LUT until splotch_plan_set_colormaps loads the plan's own (lut_buf)
    int *vlut_tab = nullptr;
    const float4 *vlut = nullptr;
    float4 *lut_buf = nullptr;
    size_t lut_cap = 0;  // entries
};

static splotch_status plan_enqueue(splotch_plan *pl, float *out, cudaStream_t st) {
    splotch_scene *sc = pl->sc;
    FrameHost &fh = pl->fh;
    FrameDev fr = frame_dev(fh, pl->fixed, pl->var);
    fr.vscale = pl->vscale;
    const size_t nvt = (size_t)fh.V * sc->n_types;
    fr.vlut = pl->vlut;
    fr.vlut_off = pl->vlut_tab;
    fr.vlut_len = pl->vlut_tab + nvt;
    CUDA_TRY(cudaMemsetAsync(pl->fixed + fh.o_counts, 0, sizeof(int) * (size_t)fh.V * fh.n_tiles, st));
    CUDA_TRY(cudaMemsetAsync(pl->fixed + fh.o_status, 0, sizeof(int) * 4, st));
    CUDA_TRY(cudaMemsetAsync(pl->fixed + fh.o_queue, 0, sizeof(int) * 4, st));
    CUDA_TRY(launch_count(sc->storage, sc->dev_view, fr, st));
    CUDA_TRY(launch_scan(fr, target_items(sc->dev, fh.T), kMinItemPairs, st));
    CUDA_TRY(launch_scatter(sc->storage, sc->dev_view, fr, (pl->rs.pr.flags & SPLOTCH_STABLE) != 0, st));
    CUDA_TRY(launch_splat(sc->dev_view, fr, (int *)(pl->fixed + fh.o_queue), out,
                          out_mode(pl->rs.pr.flags), pl->grid, st));
    CUDA_TRY(cudaMemcpyAsync(pl->box, pl->fixed + fh.o_sizes, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(pl->box + 8, pl->fixed + fh.o_status, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_destroy(splotch_plan *pl) {
    if (!pl) return SPLOTCH_OK;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    cudaDeviceSynchronize();
    if (pl->var) pl->sc->mem.release(pl->var, 0);
    if (pl->fixed) pl->sc->mem.release(pl->fixed, 0);
    if (pl->vscale) pl->sc->mem.release(pl->vscale, 0);
    if (pl->vlut_tab) pl->sc->mem.release(pl->vlut_tab, 0);
    if (pl->lut_buf) pl->sc->mem.release(pl->lut_buf, 0);
    if (pl->box) cudaFreeHost(pl->box);
    cudaStreamSynchronize(0);
    delete pl;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_create(splotch_scene *sc, const splotch_camera *cams, int32_t n_views,
                                              const splotch_render_params *params, double headroom, void *stream,
                                              splotch_plan **out) {
    if (!sc || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    if (!(headroom >= 1.0) || headroom > 100.0) return fail(SPLOTCH_ERR_INVALID_ARG, "headroom outside [1, 100]");
    cudaStream_t st = (cudaStream_t)stream;
    splotch_plan *pl = new splotch_plan();
    pl->sc = sc;
    splotch_status s = setup_views(cams, n_views, params, pl->rs);
    if (s != SPLOTCH_OK) {
        delete pl;
        return s;
    }
    pl->use_graph = (pl->rs.pr.flags & SPLOTCH_PLAN_GRAPH) != 0;
    layout_fixed(pl->fh, sc, pl->rs.V, pl->rs.views[0].n_tiles, pl->rs.T, pl->rs.pr.block_particles);
    pl->fixed = (char *)sc->mem.alloc(pl->fh.fixed_bytes, st);
    if (!pl->fixed) {
        delete pl;
        return fail(SPLOTCH_ERR_OOM, "plan workspace");
    }
    if (cudaMallocHost((void **)&pl->box, 16 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        splotch_plan_destroy(pl);
        return fail(SPLOTCH_ERR_OOM, "pinned host buffer");
    }
    int64_t sizes[8];
    s = count_and_size(sc, pl->rs, pl->fh, pl->fixed, st, sizes);
    if (s != SPLOTCH_OK) {
        splotch_plan_destroy(pl);
        return s;
    }
    const int64_t nt = (int64_t)pl->rs.V * pl->fh.n_tiles;
    const int64_t pairs = (int64_t)std::ceil((double)sizes[kSizePairs] * headroom) + 1024;
    const int64_t items = std::min<int64_t>(INT32_MAX / 2, (int64_t)std::ceil((double)sizes[kSizeItems] * headroom) + nt / 8 + 64);
    const int64_t splits = std::min<int64_t>(nt, (int64_t)std::ceil((double)sizes[kSizeSplits] * headroom) + 64);
    layout_var(pl->fh, pairs, (int)std::max<int64_t>(items, nt), (int)splits, false);
    pl->var = (char *)sc->mem.alloc(pl->fh.var_bytes, st);
    if (!pl->var) {
        splotch_plan_destroy(pl);
        return fail(SPLOTCH_ERR_OOM, "plan tile lists (%zu bytes)", pl->fh.var_bytes);
    }
    if (cudaMemsetAsync(pl->var + pl->fh.o_scratch, 0, pl->fh.var_bytes - pl->fh.o_scratch, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        splotch_plan_destroy(pl);
        return fail(SPLOTCH_ERR_CUDA, "plan scratch");
    }
    pl->grid = splat_grid(sc->dev, pl->rs.T, INT32_MAX);
    // emission scale per view and species (1 until splotch_plan_set_brightness): a fixed
    // device array, so a captured graph reads the current scales at every replay
    {
        const size_t nv = (size_t)pl->rs.V * sc->n_types;
        pl->vscale = (float *)sc->mem.alloc(sizeof(float) * nv, st);
        std::vector<float> ones(nv, 1.0f);
        if (!pl->vscale ||
            cudaMemcpyAsync(pl->vscale, ones.data(), sizeof(float) * nv, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            splotch_plan_destroy(pl);
            return fail(SPLOTCH_ERR_OOM, "plan view scales");
        }
        // every view starts with the scene's colormaps
        std::vector<int> tab(2 * nv);
        std::vector<int> off(sc->n_types), len(sc->n_types);
        cudaMemcpy(off.data(), sc->dev_view.lut_off, sizeof(int) * sc->n_types, cudaMemcpyDeviceToHost);
        cudaMemcpy(len.data(), sc->dev_view.lut_len, sizeof(int) * sc->n_types, cudaMemcpyDeviceToHost);
        for (size_t k = 0; k < nv; ++k) tab[k] = off[k % sc->n_types], tab[nv + k] = len[k % sc->n_types];
        pl->vlut_tab = (int *)sc->mem.alloc(sizeof(int) * 2 * nv, st);
        pl->vlut = sc->dev_view.lut;
        if (!pl->vlut_tab ||
            cudaMemcpyAsync(pl->vlut_tab, tab.data(), sizeof(int) * 2 * nv, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            splotch_plan_destroy(pl);
            return fail(SPLOTCH_ERR_OOM, "plan colormap table");
        }
    }
    *out = pl;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_set_cameras(splotch_plan *pl, const splotch_camera *cams, int32_t n_views,
                                                   void *stream) {
    if (!pl) return fail(SPLOTCH_ERR_INVALID_ARG, "plan is NULL");
    if (n_views != pl->rs.V) return fail(SPLOTCH_ERR_INVALID_ARG, "view count differs from the plan");
    RenderSetup rs;
    splotch_render_params pr = pl->rs.pr;
    pr.tile = pl->rs.T;
    splotch_status s = setup_views(cams, n_views, &pr, rs);
    if (s != SPLOTCH_OK) return s;
    if (rs.W != pl->rs.W || rs.H != pl->rs.H) return fail(SPLOTCH_ERR_INVALID_ARG, "image size differs from the plan");
    pl->rs.views = rs.views;
    CUDA_TRY(cudaMemcpyAsync(pl->fixed + pl->fh.o_views, pl->rs.views.data(), sizeof(ViewParams) * n_views,
                             cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_set_brightness(splotch_plan *pl, const float *scale, void *stream) {
    if (!pl) return fail(SPLOTCH_ERR_INVALID_ARG, "plan is NULL");
    const int nt = pl->sc->n_types;
    const size_t nv = (size_t)pl->rs.V * nt;
    std::vector<float> v(nv, 1.0f);
    if (scale)
        for (size_t k = 0; k < nv; ++k) {
            if (!(scale[k] >= 0.0f) || !std::isfinite(scale[k]))
                return fail(SPLOTCH_ERR_INVALID_ARG, "scale[%zu] (view %zu, species %zu) not finite and >= 0", k,
                            k / nt, k % nt);
            v[k] = scale[k];
        }
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(pl->vscale, v.data(), sizeof(float) * nv, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_set_colormaps(splotch_plan *pl, const float *const *cmap_rgb,
                                                     const int32_t *cmap_len, void *stream) {
    if (!pl) return fail(SPLOTCH_ERR_INVALID_ARG, "plan is NULL");
    splotch_scene *sc = pl->sc;
    if (sc->dev_view.emit)
        return fail(SPLOTCH_ERR_UNSUPPORTED, "per-view colormaps of a scene with vector colour (its colour is per particle)");
    const int nt = sc->n_types;
    const size_t nv = (size_t)pl->rs.V * nt;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> tab(2 * nv);
    if (!cmap_rgb) {
        // back to the scene's colormaps
        std::vector<int> off(nt), len(nt);
        CUDA_TRY(cudaMemcpy(off.data(), sc->dev_view.lut_off, sizeof(int) * nt, cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(len.data(), sc->dev_view.lut_len, sizeof(int) * nt, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < nv; ++k) tab[k] = off[k % nt], tab[nv + k] = len[k % nt];
        if (pl->vlut != sc->dev_view.lut && pl->exec) {
            cudaGraphExecDestroy(pl->exec);  // captured with the plan's LUT: capture again
            pl->exec = nullptr;
        }
        pl->vlut = sc->dev_view.lut;
    } else {
        if (!cmap_len) return fail(SPLOTCH_ERR_INVALID_ARG, "cmap_len is NULL");
        size_t total = 0;
        for (size_t k = 0; k < nv; ++k) {
            if (cmap_len[k] < 2 || cmap_len[k] > (1 << 20) || !cmap_rgb[k])
                return fail(SPLOTCH_ERR_INVALID_ARG, "colormap of view %zu, species %zu: NULL or not 2..2^20 entries",
                            k / nt, k % nt);
            for (int j = 0; j < 3 * cmap_len[k]; ++j)
                if (!std::isfinite(cmap_rgb[k][j]))
                    return fail(SPLOTCH_ERR_INVALID_ARG, "colormap of view %zu, species %zu not finite", k / nt, k % nt);
            tab[k] = (int)total;
            tab[nv + k] = cmap_len[k];
            total += (size_t)cmap_len[k];
        }
        if (total > (size_t)INT32_MAX) return fail(SPLOTCH_ERR_UNSUPPORTED, "colormaps above 2^31 entries");
        // entries premultiplied by the species brightness, as the scene's
        const std::vector<float> &bright = sc->brightness;
        std::vector<float> lut(4 * total);
        for (size_t k = 0; k < nv; ++k)
            for (int j = 0; j < cmap_len[k]; ++j) {
                float *q = &lut[4 * ((size_t)tab[k] + j)];
                for (int c = 0; c < 3; ++c) q[c] = bright[k % nt] * cmap_rgb[k][3 * j + c];
                q[3] = 0.0f;
            }
        if (total > pl->lut_cap) {
            float4 *nb = (float4 *)sc->mem.alloc(sizeof(float4) * total, st);
            if (!nb) return fail(SPLOTCH_ERR_OOM, "plan colormaps (%zu entries)", total);
            CUDA_TRY(cudaStreamSynchronize(st));  // no launch of this plan may still read the old one
            if (pl->lut_buf) sc->mem.release(pl->lut_buf, st);
            pl->lut_buf = nb;
            pl->lut_cap = total;
        }
        if (pl->vlut != pl->lut_buf && pl->exec) {
            cudaGraphExecDestroy(pl->exec);  // the captured kernels read another LUT: capture again
            pl->exec = nullptr;
        }
        pl->vlut = pl->lut_buf;
        CUDA_TRY(cudaMemcpyAsync(pl->lut_buf, lut.data(), sizeof(float) * lut.size(), cudaMemcpyHostToDevice, st));
    }
    CUDA_TRY(cudaMemcpyAsync(pl->vlut_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_launch(splotch_plan *pl, float *out, void *stream) {
    if (!pl || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (!pl->use_graph) return plan_enqueue(pl, out, st);
    if (!pl->exec || pl->exec_out != out) {
        if (pl->exec) {
            cudaGraphExecDestroy(pl->exec);
            pl->exec = nullptr;
        }
        if (!pl->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
        // one eager run sets kernel attributes outside capture
        splotch_status s = plan_enqueue(pl, out, pl->cap_stream);
        if (s != SPLOTCH_OK) return s;
        CUDA_TRY(cudaStreamSynchronize(pl->cap_stream));
        CUDA_TRY(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
        s = plan_enqueue(pl, out, pl->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
        if (s != SPLOTCH_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&pl->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        pl->exec_out = out;
    }
    CUDA_TRY(cudaGraphLaunch(pl->exec, st));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_check(splotch_plan *pl, void *stream, int64_t *pairs_needed) {
    if (!pl) return fail(SPLOTCH_ERR_INVALID_ARG, "plan is NULL");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const int64_t *sizes = pl->box;
    const int *stat = (const int *)(pl->box + 8);
    if (pairs_needed) *pairs_needed = sizes[kSizePairs];
    if (stat[kStatTimeout]) return fail(SPLOTCH_ERR_TIMEOUT, "splat stage wait timed out");
    if (stat[kStatOverflow])
        return fail(SPLOTCH_ERR_CAPACITY, "frame needs %lld pairs / %lld items / %lld split tiles, plan holds %lld / %d / %d",
                    (long long)sizes[kSizePairs], (long long)sizes[kSizeItems], (long long)sizes[kSizeSplits],
                    (long long)pl->fh.pair_cap, pl->fh.item_cap, pl->fh.split_cap);
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_plan_info(const splotch_plan *pl, int64_t *device_bytes, int32_t *tile,
                                            int64_t *pair_capacity) {
    if (!pl) return fail(SPLOTCH_ERR_INVALID_ARG, "plan is NULL");
    if (device_bytes) *device_bytes = (int64_t)(pl->fh.fixed_bytes + pl->fh.var_bytes);
    if (tile) *tile = pl->rs.T;
    if (pair_capacity) *pair_capacity = pl->fh.pair_cap;
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_selftest_bounded_wait(int64_t limit_cycles, void *stream) {
    if (limit_cycles < 1000 || limit_cycles > 10000000000LL)
        return fail(SPLOTCH_ERR_INVALID_ARG, "limit_cycles outside 1e3..1e10");
    cudaStream_t st = (cudaStream_t)stream;
    int *d = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int), st));
    cudaError_t e = launch_selftest_wait((long long)limit_cycles, d, st);
    int r = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    if (r == 2) return fail(SPLOTCH_ERR_TIMEOUT, "bounded wait gave up after %lld cycles", (long long)limit_cycles);
    if (r == 1) return SPLOTCH_OK;
    return fail(SPLOTCH_ERR_CUDA, "selftest kernel did not report");
}

extern "C" splotch_status splotch_final_transform(float *a, int64_t count, void *stream) {
    if (count < 0 || (count > 0 && !a)) return fail(SPLOTCH_ERR_INVALID_ARG, "bad buffer");
    CUDA_TRY(launch_final(a, count, (cudaStream_t)stream));
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_compose_maps(const float *maps, int32_t n_maps, int64_t pixels, float *out,
                                               void *stream) {
    if (n_maps < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "n_maps < 1");
    if (pixels < 0) return fail(SPLOTCH_ERR_INVALID_ARG, "pixels < 0");
    if (pixels > 0 && (!maps || !out)) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL buffer");
    if (pixels > INT64_MAX / (6 * (int64_t)n_maps)) return fail(SPLOTCH_ERR_INVALID_ARG, "maps too large");
    const uintptr_t m0 = (uintptr_t)maps, m1 = m0 + sizeof(float) * 6 * (uintptr_t)pixels * (uintptr_t)n_maps;
    const uintptr_t o0 = (uintptr_t)out, o1 = o0 + sizeof(float) * 6 * (uintptr_t)pixels;
    if (pixels > 0 && o0 < m1 && m0 < o1) return fail(SPLOTCH_ERR_INVALID_ARG, "out overlaps maps");
    CUDA_TRY(launch_compose_maps(maps, n_maps, pixels, out, (cudaStream_t)stream));
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// Render without allocation.  Some callers cannot allocate device memory while rendering:
// a host application that has reserved the whole GPU for its own memory manager, or a
// real-time loop whose rules forbid allocation after start-up (an allocation can block on
// the device and take memory the application has planned for).  This path keeps the
// whole frame workspace in one fixed device array declared below.  The CUDA runtime
// places that array on every GPU that loads this library, and it stays there until the
// process exits.

static constexpr size_t kStaticBytes = size_t(32) << 20;          // 32 MiB per GPU
static constexpr int64_t kStaticRelBudget = int64_t(2) << 20;      // chunk bases: 2 MiB of it
static constexpr int kStaticSplits = 256;                          // split-tile scratch slots
static constexpr size_t kStaticSplitBytes = size_t(8) << 20;       // and at most 8 MiB for them
static constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

static std::mutex g_static_mu;
static void *g_static_addr[kMaxDevices];  // device address of g_static_ws, per device

// Device address of the fixed workspace on the current device.  Host code cannot use the
// symbol's own name as a device pointer, so it asks the runtime once per device, with that
// device current; later calls reuse the address.
static splotch_status static_workspace(int dev, char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(SPLOTCH_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p)
            return fail(SPLOTCH_ERR_CUDA, "cudaGetSymbolAddress of the fixed workspace: %s", cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = static_cast<char *>(g_static_addr[dev]);
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_render_noalloc(splotch_scene *sc, const splotch_camera *cam,
                                                 const splotch_render_params *params, float *out, void *stream) {
    if (!sc || !cam || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    splotch_render_params pr = params ? *params : splotch_default_params();
    splotch_status s = check_params(&pr);
    if (s != SPLOTCH_OK) return s;
    if (cam->width < 1 || cam->height < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "image size < 1");
    if ((int64_t)cam->width * cam->height > (int64_t)1 << 30) return fail(SPLOTCH_ERR_UNSUPPORTED, "image larger than 2^30 px");
    int T = 0;
    s = choose_tile(cam->width, cam->height, pr.tile, &T);
    if (s != SPLOTCH_OK) return s;
    ViewParams vp;
    s = make_view(cam, pr, T, vp);
    if (s != SPLOTCH_OK) return s;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    // the scene's arrays live on the device it was created on, and the fixed array used
    // below is the current device's: both must be the same GPU
    if (dev != sc->dev)
        return fail(SPLOTCH_ERR_INVALID_ARG, "current device %d is not the scene's device %d", dev, sc->dev);
    char *base = nullptr;
    s = static_workspace(dev, &base);
    if (s != SPLOTCH_OK) return s;

    // carve the fixed array: per-tile tables, then tile lists and split-tile scratch
    FrameHost fh;
    layout_fixed(fh, sc, 1, vp.n_tiles, T, pr.block_particles, kStaticRelBudget);
    const size_t fixed = align256(fh.fixed_bytes);
    const int splits = (int)std::min<size_t>(std::min(vp.n_tiles, kStaticSplits),
                                             std::max<size_t>(1, kStaticSplitBytes / split_scratch_bytes(T)));
    const size_t scratch = align256(split_scratch_bytes(T) * splits) + align256(sizeof(int) * splits);
    if (fixed + scratch + 4096 > kStaticBytes)
        return fail(SPLOTCH_ERR_UNSUPPORTED, "%d tiles of %d px need %zu bytes of tables, more than the %zu-byte fixed workspace",
                    vp.n_tiles, T, fixed + scratch, kStaticBytes);
    const int64_t pairs = (int64_t)((kStaticBytes - fixed - scratch - 1024) / sizeof(float4));
    layout_var(fh, pairs, INT32_MAX, splits, false, false);
    if (fixed + fh.var_bytes > kStaticBytes)
        return fail(SPLOTCH_ERR_UNSUPPORTED, "fixed workspace layout overflow");
    char *var = base + fixed;
    FrameDev fr = frame_dev(fh, base, var);

    // every call shares the array: zero what the kernels count into before they start
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(base + fh.o_views, &vp, sizeof(ViewParams), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(base + fh.o_counts, 0, sizeof(int) * (size_t)vp.n_tiles, st));
    CUDA_TRY(cudaMemsetAsync(base + fh.o_status, 0, sizeof(int) * 4, st));
    CUDA_TRY(cudaMemsetAsync(base + fh.o_queue, 0, sizeof(int) * 4, st));
    CUDA_TRY(cudaMemsetAsync(var + fh.o_scratch, 0, fh.var_bytes - fh.o_scratch, st));
    CUDA_TRY(launch_count(sc->storage, sc->dev_view, fr, st));
    CUDA_TRY(launch_scan(fr, target_items(sc->dev, T), kMinItemPairs, st));
    CUDA_TRY(launch_scatter(sc->storage, sc->dev_view, fr, (pr.flags & SPLOTCH_STABLE) != 0, st));
    CUDA_TRY(launch_splat(sc->dev_view, fr, (int *)(base + fh.o_queue), out,
                          out_mode(pr.flags), sm_count(dev) * std::max(1, splat_blocks_per_sm(T)), st));
    int64_t sizes[8];
    int stat[4];
    CUDA_TRY(cudaMemcpyAsync(sizes, base + fh.o_sizes, sizeof(sizes), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(stat, base + fh.o_status, sizeof(stat), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (stat[kStatTimeout]) return fail(SPLOTCH_ERR_TIMEOUT, "splat stage wait timed out");
    if (stat[kStatOverflow])
        return fail(SPLOTCH_ERR_CAPACITY,
                    "frame needs %lld particle-tile pairs and %lld split tiles; the fixed %zu-byte workspace holds %lld and %d",
                    (long long)sizes[kSizePairs], (long long)sizes[kSizeSplits], kStaticBytes, (long long)pairs, splits);
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// Out-of-core render: the particle set stays in host memory and is rendered in chunks.
// Section 3.1 moves data sets larger than the coprocessor's memory through it in
// double-buffered pieces, transfers overlapping work; here the
// accumulation is a sum over particles in absorption = emission mode (Section 2.1), so
// chunks add into one image and the final transform runs once.  While chunk k renders on
// the caller's stream, chunk k + 1 is prepared on a second stream (read in place from
// page-locked host memory, or staged), so the host-to-device transfer overlaps the render.

// Exact per-species range of the (logged) intensity over the whole set, chunk by chunk.
// Joint min / max keys of `comps`-component field values over the species with use[t],
// read chunk by chunk (through a device-visible address when the field is device or
// page-locked memory, else staged).
static cudaError_t field_ranges(const splotch_scene_desc *d, const float *field, int comps, const std::vector<int> &use,
                                int64_t chunk, cudaStream_t st, Mem &mem, unsigned *keys) {
    cudaPointerAttributes pa{};
    bool direct = d->on_device != 0;
    const float *dev_in = field;
    if (!direct && cudaPointerGetAttributes(&pa, field) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer) {
        direct = true;
        dev_in = (const float *)pa.devicePointer;
    }
    cudaGetLastError();
    float *stage = nullptr;
    if (!direct) {
        stage = (float *)mem.alloc(sizeof(float) * comps * (size_t)std::min<int64_t>(chunk, d->n), st);
        if (!stage) return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaSuccess;
    for (int64_t b = 0; b < d->n && e == cudaSuccess; b += chunk) {
        const int64_t len = std::min(chunk, d->n - b);
        const float *src = dev_in + comps * b;
        if (!direct) {
            e = cudaMemcpyAsync(stage, field + comps * b, sizeof(float) * comps * len, cudaMemcpyHostToDevice, st);
            src = stage;
        }
        for (int t = 0; t < d->n_types && e == cudaSuccess; ++t) {
            const int64_t a0 = std::max(b, d->type_begin[t]), a1 = std::min(b + len, d->type_begin[t + 1]);
            if (use[t] && a1 > a0)
                e = launch_minmax(0, src - comps * b, comps * a0, comps * a1, d->i_log[t], keys + 2 * t, st);
        }
        if (!direct && e == cudaSuccess) e = cudaStreamSynchronize(st);  // staging reused
    }
    if (stage) mem.release(stage, st);
    return e;
}

// Per-species ranges over the whole set (given, or the joint min / max of the intensity,
// or of the colour components for vector-coloured species), so every chunk normalises alike.
static splotch_status streamed_ranges(const splotch_scene_desc *d, int64_t chunk, cudaStream_t st, Mem &mem,
                                      std::vector<float> &lo, std::vector<float> &hi) {
    lo.assign(d->n_types, 0.0f);
    hi.assign(d->n_types, 0.0f);
    if (d->i_min) {
        for (int t = 0; t < d->n_types; ++t) lo[t] = d->i_min[t], hi[t] = d->i_max[t];
        return SPLOTCH_OK;
    }
    unsigned *keys = (unsigned *)mem.alloc(align256(sizeof(unsigned) * 2 * d->n_types), st);
    if (!keys) return fail(SPLOTCH_ERR_OOM, "range staging");
    std::vector<unsigned> init(2 * d->n_types);
    for (int t = 0; t < d->n_types; ++t) init[2 * t] = 0xFFFFFFFFu, init[2 * t + 1] = 0u;
    std::vector<int> scalar(d->n_types, 1), vector(d->n_types, 0);
    bool any_vec = false;
    for (int t = 0; d->col_vector && t < d->n_types; ++t)
        if (d->col_vector[t]) scalar[t] = 0, vector[t] = 1, any_vec = true;
    cudaError_t e = cudaMemcpyAsync(keys, init.data(), sizeof(unsigned) * init.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = field_ranges(d, d->intensity, 1, scalar, chunk, st, mem, keys);
    if (e == cudaSuccess && any_vec) e = field_ranges(d, d->rgb, 3, vector, chunk, st, mem, keys);
    if (e == cudaSuccess) e = cudaMemcpyAsync(init.data(), keys, sizeof(unsigned) * init.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mem.release(keys, st);
    if (e == cudaErrorMemoryAllocation) return fail(SPLOTCH_ERR_OOM, "range staging");
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "intensity range: %s", cudaGetErrorString(e));
    for (int t = 0; t < d->n_types; ++t) {
        lo[t] = init[2 * t] == 0xFFFFFFFFu ? 0.0f : order_key_inv(init[2 * t]);
        hi[t] = init[2 * t + 1] == 0u ? 0.0f : order_key_inv(init[2 * t + 1]);
    }
    return SPLOTCH_OK;
}

extern "C" splotch_status splotch_render_streamed(const splotch_scene_desc *d, int64_t chunk,
                                                  const splotch_camera *cam, const splotch_render_params *params,
                                                  float *out, void *stream) {
    if (!d || !cam || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    if (chunk < 1) return fail(SPLOTCH_ERR_INVALID_ARG, "chunk < 1");
    splotch_status s = validate_desc(d);
    if (s != SPLOTCH_OK) return s;
    splotch_render_params pr = params ? *params : splotch_default_params();
    s = check_params(&pr);
    if (s != SPLOTCH_OK) return s;
    const bool keep_accum = (pr.flags & SPLOTCH_OUT_ACCUM) != 0;
    const bool add = (pr.flags & SPLOTCH_OUT_ADD) != 0;
    pr.flags = (pr.flags & ~(SPLOTCH_SYNC | SPLOTCH_TIMING | SPLOTCH_OUT_ACCUM)) | SPLOTCH_OUT_ADD;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    Mem mem;
    mem.a = d->allocator;
    mem.dev = dev;
    std::vector<float> lo, hi;
    s = streamed_ranges(d, chunk, st, mem, lo, hi);
    if (s != SPLOTCH_OK) return s;
    const size_t img = sizeof(float) * 3 * (size_t)cam->width * (size_t)cam->height;
    if (!add) CUDA_TRY(cudaMemsetAsync(out, 0, img, st));

    cudaStream_t side = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    // the previous chunk's scene and frame are released only once its render is ordered
    // behind this one
    splotch_scene *prev = nullptr;
    splotch_frame *prevf = nullptr;
    auto drop = [&](splotch_scene *sc) {
        if (!sc) return;
        sc->mem.release(sc->attr, st);
        sc->mem.release(sc->meta, st);
        delete sc;
    };
    const float *src[5] = {d->x, d->y, d->z, d->h, d->intensity};
    // chunk sizes ramp up from a sixth of `chunk` by 3/2 per chunk: the first transfer,
    // which nothing can hide, is short, and each later one overlaps the render of a chunk
    // two thirds its size.  The host link moves FP32 attributes about 1.4x faster than a
    // frame of the two-species benchmark renders them, so a faster ramp leaves the render
    // waiting for its data, and a slower one adds chunks, each with its own kernel tails.
    int64_t step = std::max<int64_t>(1, std::min(chunk, std::max<int64_t>(chunk / 6, (int64_t)1 << 20)));
    for (int64_t b = 0, len = 0; b < d->n && s == SPLOTCH_OK; b += len, step = std::min(chunk, step + step / 2)) {
        len = std::min(step, d->n - b);
        splotch_scene_desc cd = *d;
        cd.n = len;
        const float *const *p = src;
        cd.x = p[0] + b, cd.y = p[1] + b, cd.z = p[2] + b, cd.h = p[3] + b, cd.intensity = p[4] + b;
        cd.rgb = d->rgb ? d->rgb + 3 * b : nullptr;
        std::vector<int64_t> tb(d->n_types + 1);
        for (int t = 0; t <= d->n_types; ++t) tb[t] = std::min(std::max(d->type_begin[t] - b, (int64_t)0), len);
        cd.type_begin = tb.data();
        cd.i_min = lo.data();
        cd.i_max = hi.data();
        cd.stream = side;
        // copied, prepared and counted (the count phase of a two-phase frame) on the side
        // stream while the previous chunk's scatter and splat run on `stream`; the host
        // waits only for the side stream.  (Scattering on the side stream as well was
        // slower: a scatter CTA needs a whole SM's registers, so it cannot start beside
        // the splat's resident CTAs.)
        splotch_scene *sc = nullptr;
        s = create_scene_impl(&cd, &sc, true);
        if (s != SPLOTCH_OK) break;
        splotch_frame *f = nullptr;
        s = splotch_frame_prepare(sc, cam, &pr, side, &f, nullptr, nullptr, nullptr);
        if (s != SPLOTCH_OK) {
            drop(sc);
            break;
        }
        s = frame_scatter(f, st);
        if (s == SPLOTCH_OK) s = frame_splat(f, out, st);
        splotch_frame_destroy(prevf);
        drop(prev);
        prev = sc;
        prevf = f;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && s == SPLOTCH_OK) s = fail(SPLOTCH_ERR_CUDA, "streamed render");
    splotch_frame_destroy(prevf);
    drop(prev);
    cudaStreamDestroy(side);
    if (s != SPLOTCH_OK) return s;
    if (!keep_accum && !add) {
        CUDA_TRY(launch_final(out, (int64_t)img / sizeof(float), st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// Test hook for the radix sort the depth-ordered render uses.
extern "C" splotch_status splotch_debug_sort(void *keys, int32_t key_bytes, uint32_t *vals, int64_t n,
                                             int32_t bit_lo, int32_t bit_hi, void *stream) {
    if (n < 0 || (n > 0 && (!keys || !vals))) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL buffer or n < 0");
    if (key_bytes != 4 && key_bytes != 8) return fail(SPLOTCH_ERR_INVALID_ARG, "key_bytes %d not 4 or 8", key_bytes);
    if (bit_lo < 0 || bit_hi > 8 * key_bytes || bit_lo > bit_hi || (bit_hi - bit_lo) % 8 != 0)
        return fail(SPLOTCH_ERR_INVALID_ARG, "key bits [%d, %d) not a whole number of bytes in [0, %d)", bit_lo,
                    bit_hi, 8 * key_bytes);
    if (n > (int64_t)UINT32_MAX) return fail(SPLOTCH_ERR_UNSUPPORTED, "more than 2^32 pairs");
    if (n <= 1) return SPLOTCH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    Mem mem;
    mem.dev = dev;
    const size_t kb = align256((size_t)key_bytes * (size_t)n), vb = align256(sizeof(uint32_t) * (size_t)n);
    char *buf = (char *)mem.alloc(kb + vb + sort_temp_bytes(n), st);
    if (!buf) return fail(SPLOTCH_ERR_OOM, "sort buffers");
    bool alt = false;
    cudaError_t e =
        key_bytes == 8
            ? radix_sort_pairs((uint64_t *)keys, (uint64_t *)buf, vals, (uint32_t *)(buf + kb), n, bit_lo, bit_hi,
                               buf + kb + vb, st, &alt)
            : radix_sort_pairs((uint32_t *)keys, (uint32_t *)buf, vals, (uint32_t *)(buf + kb), n, bit_lo, bit_hi,
                               buf + kb + vb, st, &alt);
    if (e == cudaSuccess && alt) {
        e = cudaMemcpyAsync(keys, buf, (size_t)key_bytes * (size_t)n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, buf + kb, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mem.release(buf, st);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "sort: %s", cudaGetErrorString(e));
    return SPLOTCH_OK;
}

// -----------------------------------------------------------------------------------------
// Depth-ordered render (absorption != emission).  Section 2.1 solves the radiative-transfer
// equation along each line of sight; with absorption A = s_t x emission per species the
// particles' updates do not commute, so every tile list is put in depth order (farthest
// first) before the splat: the scatter writes a (tile, depth) key per record, a stable
// radix sort orders the keys, and the records are gathered in that order.
extern "C" splotch_status splotch_render_ordered(splotch_scene *sc, const splotch_camera *cam,
                                                 const splotch_render_params *params, const float *absorb,
                                                 float *out, void *stream) {
    if (!sc || !cam || !absorb || !out) return fail(SPLOTCH_ERR_INVALID_ARG, "NULL argument");
    for (int t = 0; t < sc->n_types; ++t)
        if (!(absorb[t] >= 0.0f) || !std::isfinite(absorb[t]))
            return fail(SPLOTCH_ERR_INVALID_ARG, "absorb[%d] not finite and >= 0", t);
    RenderSetup rs;
    splotch_status s = setup_views(cam, 1, params, rs);
    if (s != SPLOTCH_OK) return s;
    if (rs.T > 32) return fail(SPLOTCH_ERR_UNSUPPORTED, "depth-ordered render: tile %d above 32 px", rs.T);
    cudaStream_t st = (cudaStream_t)stream;
    const int split = ordered_split(rs.T);
    const int target = std::max(1, sm_count(sc->dev) * ordered_workers_per_sm() * 4 / (split * split));
    FrameHost fh;
    layout_fixed(fh, sc, 1, rs.views[0].n_tiles, rs.T, rs.pr.block_particles);
    char *fixed = (char *)sc->mem.alloc(fh.fixed_bytes, st);
    if (!fixed) return fail(SPLOTCH_ERR_OOM, "frame workspace (%zu bytes)", fh.fixed_bytes);
    int64_t sizes[8];
    s = count_and_size(sc, rs, fh, fixed, st, sizes, nullptr, target);
    if (s != SPLOTCH_OK) {
        sc->mem.release(fixed, st);
        return s;
    }
    const int64_t P = sizes[kSizePairs];
    const int items = (int)sizes[kSizeItems], splits = (int)sizes[kSizeSplits];
    if (P > (int64_t)UINT32_MAX) {
        sc->mem.release(fixed, st);
        return fail(SPLOTCH_ERR_UNSUPPORTED, "depth-ordered render: more than 2^32 particle-tile pairs");
    }
    layout_var(fh, P, items, splits, false);
    // depth-ordered binning buffers: per particle (n) and per pair (P)
    const int64_t n = std::max<int64_t>(1, sc->n), Pm = std::max<int64_t>(1, P);
    Carve cv;
    const size_t o_prec = cv.take(sizeof(float4) * (size_t)n);
    const size_t o_srec = cv.take(sizeof(float4) * (size_t)n);
    const size_t o_dk0 = cv.take(sizeof(uint32_t) * (size_t)n);
    const size_t o_dk1 = cv.take(sizeof(uint32_t) * (size_t)n);
    const size_t o_id0 = cv.take(sizeof(uint32_t) * (size_t)n);
    const size_t o_id1 = cv.take(sizeof(uint32_t) * (size_t)n);
    const size_t o_cnt = cv.take(sizeof(uint32_t) * (size_t)(n + 1));
    const size_t o_rec = cv.take(sizeof(float4) * (size_t)Pm);
    const size_t o_tk0 = cv.take(sizeof(uint32_t) * (size_t)Pm);
    const size_t o_tk1 = cv.take(sizeof(uint32_t) * (size_t)Pm);
    const size_t o_tv0 = cv.take(sizeof(uint32_t) * (size_t)Pm);
    const size_t o_tv1 = cv.take(sizeof(uint32_t) * (size_t)Pm);
    const size_t o_map = cv.take(sizeof(float) * 6 * (size_t)rs.T * rs.T * (size_t)std::max(1, items));
    const size_t o_abs = cv.take(sizeof(float) * (size_t)sc->n_types);
    const size_t o_tmp = cv.take(std::max(sort_temp_bytes(std::max(n, Pm) + 1), scan_temp_bytes(n + 1)));
    const size_t o_kr = cv.take(sizeof(uint32_t) * 2);
    char *var = (char *)sc->mem.alloc(fh.var_bytes, st);
    char *ex = var ? (char *)sc->mem.alloc(cv.off, st) : nullptr;
    if (!var || !ex) {
        if (var) sc->mem.release(var, st);
        sc->mem.release(fixed, st);
        return fail(SPLOTCH_ERR_OOM, "ordered render workspace (%zu + %zu bytes)", fh.var_bytes, cv.off);
    }
    cudaError_t e = cudaMemsetAsync(var + fh.o_scratch, 0, fh.var_bytes - fh.o_scratch, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(fixed + fh.o_queue, 0, sizeof(int) * 4, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ex + o_abs, absorb, sizeof(float) * sc->n_types, cudaMemcpyHostToDevice, st);
    FrameDev fr = frame_dev(fh, fixed, var);
    // particles in depth order (stable from index order: equal depths keep index order)
    uint32_t *dka = (uint32_t *)(ex + o_dk0), *dkb = (uint32_t *)(ex + o_dk1);
    uint32_t *ida = (uint32_t *)(ex + o_id0), *idb = (uint32_t *)(ex + o_id1);
    bool alt = false;
    uint32_t *krange = (uint32_t *)(ex + o_kr);
    if (e == cudaSuccess) e = cudaMemsetAsync(krange, 0xFF, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(krange + 1, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess)
        e = launch_depth_records(sc->storage, sc->dev_view, fr.views, (float4 *)(ex + o_prec), dka, ida, krange, st);
    // sort only the bits the active depth keys span (relative to the smallest)
    uint32_t kr[2] = {1u, 0u};
    if (e == cudaSuccess) e = cudaMemcpyAsync(kr, krange, sizeof(kr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int dbits = 32;
    uint32_t inactive = 0xFFFFFFFFu;  // the key of a particle that is not active
    if (e == cudaSuccess && kr[0] <= kr[1] && kr[1] - kr[0] < 0xFFFFFFFEu) {
        const uint32_t span = kr[1] - kr[0];
        inactive = span + 1u;
        dbits = 8;
        while (dbits < 32 && ((uint64_t)span + 1u) >> dbits) dbits += 8;
        e = launch_rebase_keys(dka, sc->n, kr[0], span, st);
    }
    if (e == cudaSuccess) e = radix_sort_pairs(dka, dkb, ida, idb, sc->n, 0, dbits, ex + o_tmp, st, &alt);
    if (alt) std::swap(dka, dkb), std::swap(ida, idb);
    // each particle's records at the scanned offsets of its tile counts, keyed by tile
    uint32_t *cnt = (uint32_t *)(ex + o_cnt);
    if (e == cudaSuccess)
        e = launch_sorted_counts(fr.views, (const float4 *)(ex + o_prec), dka, ida, sc->n, inactive,
                                 (float4 *)(ex + o_srec), cnt, st);
    if (e == cudaSuccess) e = exclusive_scan_u32(cnt, sc->n + 1, ex + o_tmp, st);
    uint32_t *tka = (uint32_t *)(ex + o_tk0), *tkb = (uint32_t *)(ex + o_tk1);
    uint32_t *tva = (uint32_t *)(ex + o_tv0), *tvb = (uint32_t *)(ex + o_tv1);
    if (e == cudaSuccess)
        e = launch_expand(fr.views, (const float4 *)(ex + o_srec), cnt, sc->n, P, (float4 *)(ex + o_rec), tka, tva,
                          fr.status, st);
    // stable by tile id: every tile list keeps depth order
    int tbits = 8;
    while (tbits < 32 && ((int64_t)(rs.views[0].n_tiles - 1) >> tbits) > 0) tbits += 8;
    if (e == cudaSuccess)
        e = radix_sort_gather(tka, tkb, tva, tvb, P, 0, tbits, ex + o_tmp, (const float4 *)(ex + o_rec), fr.lists, st);
    const int64_t squares = (int64_t)std::max(1, items) * split * split;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count(sc->dev) * ordered_ctas_per_sm(),
                                                                (squares + 3) / 4));
    if (e == cudaSuccess)
        e = launch_splat_ordered(sc->dev_view, fr, (int *)(fixed + fh.o_queue), out, (const float *)(ex + o_abs),
                                 (float *)(ex + o_map), (rs.pr.flags & SPLOTCH_OUT_MAP) ? 1 : 0, grid, st);
    int stat[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(stat, fixed + fh.o_status, sizeof(stat), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    sc->mem.release(ex, st);
    sc->mem.release(var, st);
    sc->mem.release(fixed, st);
    if (e != cudaSuccess) return fail(SPLOTCH_ERR_CUDA, "ordered render: %s", cudaGetErrorString(e));
    if (stat[kStatOverflow]) return fail(SPLOTCH_ERR_CUDA, "depth-ordered binning: tile counts disagree");
    if (stat[kStatTimeout]) return fail(SPLOTCH_ERR_TIMEOUT, "splat stage wait timed out");
    return SPLOTCH_OK;
}
