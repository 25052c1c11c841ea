/*
 * Splotch rendering oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the Splotch hot path
 * computes (Dykes et al., "Splotch: porting and optimizing for the Xeon Phi").
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline
 * leg may load this file.  It shares no code with the CUDA library.
 *
 * Precision.  Values (colours, Gaussian weights, accumulation, final
 * transform) are FP64.  Every comparison that turns floating point into an
 * integer (near-plane cull, pixel bounding box, pixel coverage, tile
 * membership, reduced-precision storage codes) is taken in FP32, the paper's
 * single precision (Section 2.1: colours and attributes are single-precision
 * floats), each operation rounded once to nearest-even with no contraction
 * (build with -ffp-contract=off).  The FP32 steps are listed in full beside
 * each function.
 *
 * Readings where the paper is silent (each one is stated where it is used):
 * right-handed camera with up projected out of the view direction; vertical
 * field of view; pixel centres at +0.5 with row 0 at the top; screen radius
 * r = F h / z_c; support radius R = max(0.75 r, 0.75 px); Gaussian sigma = R/2
 * truncated at d < R; linear colormap interpolation; emission = absorption
 * with final transform 1 - exp(-a); strict "<" at both thresholds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------------
 * Camera (Section 2.1: positions are roto-translated and perspective-projected with
 * reference to the supplied camera and look-at positions; Section 3.1: the transform
 * parameters are computed once per frame).
 *
 * FP64, each operation rounded once, in this order:
 *   d = L - E;  f = d / |d|;  s' = f x U;  s = s' / |s'|;  u = s x f
 *   rows of the 3x4 matrix: (s, -(s.E)), (u, -(u.E)), (f, -(f.E))
 *   F = (0.5 H) / tan(fov_deg * (pi/360))        (vertical field of view)
 * then each entry rounded once to FP32.  p = {F, W/2, H/2, z_near} in FP32.
 * Rejected: W or H < 1, fov outside (0, 180), z_near <= 0, E == L, |s'| <= 1e-9 |U|.
 * ------------------------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3])
{
    double t = a[0] * b[0];
    t = t + a[1] * b[1];
    t = t + a[2] * b[2];
    return t;
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

int orc_camera(const double eye[3], const double look[3], const double up[3], double fov_deg,
               double z_near, double z_far, int W, int H, float m[12], float p[5])
{
    if (W < 1 || H < 1 || !(fov_deg > 0.0 && fov_deg < 180.0) || !(z_near > 0.0)) return ORC_EINVAL;
    const int has_far = z_far > 0.0 && isfinite(z_far);
    if (has_far && !(z_far > z_near)) return ORC_EINVAL;
    double d[3] = {look[0] - eye[0], look[1] - eye[1], look[2] - eye[2]};
    double nd = sqrt(dot3(d, d));
    if (!(nd > 0.0)) return ORC_EINVAL;
    double f[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
    double s0[3];
    cross3(f, up, s0);
    double ns = sqrt(dot3(s0, s0));
    double nu = sqrt(dot3(up, up));
    if (!(ns > 1e-9 * nu)) return ORC_EINVAL;
    double s[3] = {s0[0] / ns, s0[1] / ns, s0[2] / ns};
    double u[3];
    cross3(s, f, u);
    const double *rows[3] = {s, u, f};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) m[4 * r + c] = (float)rows[r][c];
        m[4 * r + 3] = (float)(-dot3(rows[r], eye));
    }
    double F = (0.5 * (double)H) / tan(fov_deg * (M_PI / 360.0));
    p[0] = (float)F;
    p[1] = 0.5f * (float)W;
    p[2] = 0.5f * (float)H;
    p[3] = (float)z_near;
    p[4] = has_far ? (float)z_far : INFINITY;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Reduced-precision storage codes (FP16 / BF16, round to nearest even), written from the
 * IEEE 754 binary16 and bfloat16 formats: the value is rounded to the nearest multiple of
 * its binade's quantum 2^(e - mantissa bits) (subnormal quantum below the smallest normal),
 * ties to even, overflow to infinity.  Exact in FP64: scaling by powers of two and rint().
 * ------------------------------------------------------------------------------------------ */
static double quantise(double v, int mant_bits, int emin, double maxfin)
{
    if (v == 0.0 || !isfinite(v)) return v;
    double a = fabs(v);
    int e;
    frexp(a, &e);            /* a = m 2^e, m in [0.5, 1): leading bit weight 2^(e-1) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    double q = ldexp(1.0, lead - mant_bits);
    double r = rint(a / q) * q; /* rint rounds half to even in the default mode */
    if (r > maxfin) r = INFINITY;
    return v < 0 ? -r : r;
}

double orc_to_f16(double v) { return quantise(v, 10, -14, 65504.0); }
double orc_to_bf16(double v) { return quantise(v, 7, -126, 3.3895313892515355e38); }

/* storage: 0 = FP32, 1 = FP16, 2 = BF16 */
static float store_f32(float v, int storage)
{
    if (storage == 1) return (float)orc_to_f16((double)v);
    if (storage == 2) return (float)orc_to_bf16((double)v);
    return v;
}

void orc_quantise_f32(int64_t n, const float *in, float *out, int storage)
{
    for (int64_t i = 0; i < n; ++i) out[i] = store_f32(in[i], storage);
}

/* ------------------------------------------------------------------------------------------
 * Preprocessing (Section 2.1: ranging, normalisation, optional logarithm of input fields).
 *   I' = ln(max(I, 1e-30)) if i_log else I;   I~ = clamp((I' - i_min) / (i_max - i_min), 0, 1)
 *   i_min / i_max: given, or the exact min / max of I' over the species when range_given = 0.
 *   A range with i_max <= i_min maps every particle to 0.
 * FP64.  For reduced-precision storage I~ is rounded to FP32, then to the storage code.
 * ------------------------------------------------------------------------------------------ */
void orc_normalise(int64_t n, const float *I, int i_log, int range_given, double i_min, double i_max,
                   int storage, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = (double)I[i];
        out[i] = i_log ? log(v > 1e-30 ? v : 1e-30) : v;
    }
    if (!range_given) {
        i_min = INFINITY;
        i_max = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            if (out[i] < i_min) i_min = out[i];
            if (out[i] > i_max) i_max = out[i];
        }
    }
    double span = i_max - i_min;
    for (int64_t i = 0; i < n; ++i) {
        double t = span > 0.0 ? (out[i] - i_min) / span : 0.0;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        if (storage != 0) t = (double)store_f32((float)t, storage);
        out[i] = t;
    }
}

/* ------------------------------------------------------------------------------------------
 * Rasterisation of one particle (Section 2.1: roto-translation, perspective projection,
 * clipping; Section 2.1: the affected area depends on the particle radius).
 *
 * FP32, each operation rounded once, left to right:
 *   xc = ((m0 x + m1 y) + m2 z) + m3,  yc and zc likewise with rows 1 and 2
 *   visible iff zn < zc <= zf (zf: the far plane, +infinity when there is none)
 *   X = cx + (F xc) / zc;  Y = cy - (F yc) / zc;  r = (F h) / zc
 *   R = rfac r, raised to rmin when below it
 *   active iff visible, X, Y, R finite, and the pixel box below is not empty
 *   box: xl = (X - R) - 0.5, xh = (X + R) - 0.5, each clamped to [-2, W + 1];
 *        i0 = max(0, ceil(xl) - 1), i1 = min(W - 1, floor(xh) + 1); rows likewise with Y, H.
 * The box is one pixel wider than the support on each side so that it contains every
 * covered pixel whatever the rounding; coverage itself is decided per pixel below.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    float X, Y, R, zc, r;
    int i0, i1, j0, j1;
    int active;
} orc_px;

static void raster_one(float x, float y, float z, float h, const float m[12], const float p[5],
                       int W, int H, float rfac, float rmin, orc_px *o)
{
    float xc = ((m[0] * x + m[1] * y) + m[2] * z) + m[3];
    float yc = ((m[4] * x + m[5] * y) + m[6] * z) + m[7];
    float zc = ((m[8] * x + m[9] * y) + m[10] * z) + m[11];
    float F = p[0], cx = p[1], cy = p[2], zn = p[3], zf = p[4];
    memset(o, 0, sizeof(*o));
    o->zc = zc;
    o->i0 = o->j0 = 0;
    o->i1 = o->j1 = -1;
    if (!(zc > zn) || !(zc <= zf)) return;
    float X = cx + (F * xc) / zc;
    float Y = cy - (F * yc) / zc;
    float r = (F * h) / zc;
    float R = rfac * r;
    if (!(R > rmin)) R = rmin;
    o->X = X;
    o->Y = Y;
    o->R = R;
    o->r = r;
    if (!(isfinite(X) && isfinite(Y) && isfinite(R))) return;
    float xl = (X - R) - 0.5f, xh = (X + R) - 0.5f;
    float yl = (Y - R) - 0.5f, yh = (Y + R) - 0.5f;
    float wmax = (float)W + 1.0f, hmax = (float)H + 1.0f;
    xl = xl < -2.0f ? -2.0f : (xl > wmax ? wmax : xl);
    xh = xh < -2.0f ? -2.0f : (xh > wmax ? wmax : xh);
    yl = yl < -2.0f ? -2.0f : (yl > hmax ? hmax : yl);
    yh = yh < -2.0f ? -2.0f : (yh > hmax ? hmax : yh);
    int i0 = (int)ceilf(xl) - 1, i1 = (int)floorf(xh) + 1;
    int j0 = (int)ceilf(yl) - 1, j1 = (int)floorf(yh) + 1;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    if (i1 > W - 1) i1 = W - 1;
    if (j1 > H - 1) j1 = H - 1;
    o->i0 = i0;
    o->i1 = i1;
    o->j0 = j0;
    o->j1 = j1;
    o->active = (i0 <= i1 && j0 <= j1);
}

/* Pixel coverage (Section 2.1: Gaussian kernel over the area the radius influences).
 * FP32: dx = (i + 0.5) - X, dy = (j + 0.5) - Y, d2 = dx dx + dy dy; covered iff d2 < R R. */
static int covered(const orc_px *o, int i, int j)
{
    float dx = ((float)i + 0.5f) - o->X;
    float dy = ((float)j + 0.5f) - o->Y;
    float d2 = dx * dx + dy * dy;
    return d2 < o->R * o->R;
}

/* Colour from a scalar through a runtime colormap (Section 2.1), linear interpolation:
 *   f = I~ (n - 1), k = min(floor f, n - 2), tau = f - k,
 *   e = beta ((1 - tau) C[k] + tau C[k+1]).   FP64. */
static void colour(double It, const float *cmap, int n, double beta, double e[3])
{
    double f = It * (double)(n - 1);
    int k = (int)floor(f);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double tau = f - (double)k;
    for (int c = 0; c < 3; ++c)
        e[c] = beta * ((1.0 - tau) * (double)cmap[3 * k + c] + tau * (double)cmap[3 * (k + 1) + c]);
}

/* Colour directly from a vector input field (Section 2.1: the RGB triple of a particle,
 * its three components ranged and normalised like a scalar, one range per species):
 *   e = beta (r~, g~, b~).   FP64. */
static void colour_vector(const double rgb[3], double beta, double e[3])
{
    for (int c = 0; c < 3; ++c) e[c] = beta * rgb[c];
}

/* Gaussian weight, sigma = sigma_over_R * R, FP64 distance from the FP32 centre. */
static double weight(const orc_px *o, int i, int j, double sor)
{
    double dx = ((double)i + 0.5) - (double)o->X;
    double dy = ((double)j + 0.5) - (double)o->Y;
    double sg = sor * (double)o->R;
    return exp(-(dx * dx + dy * dy) / (sg * sg));
}

/* ------------------------------------------------------------------------------------------
 * Scene block shared by the entry points below: particles (FP32 SoA, already quantised
 * for reduced-precision storage by the caller through orc_quantise_f32), normalised
 * intensities (FP64), species ranges, colormaps, brightness and the camera.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const float *x, *y, *z, *h;
    const double *It;
    int n_types;
    const int64_t *type_begin;
    const float *const *cmap;
    const int *cmap_len;
    const double *beta;
    float m[12], p[5];
    int W, H;
    float rfac, rmin;
    double sor;
    const double *rgb;  /* n x 3 normalised colour components, or NULL */
    const int *vec;     /* per species: 1 = colour from rgb, or NULL (all from the colormap) */
} orc_scene;

static int type_of(const orc_scene *s, int64_t i)
{
    int t = 0;
    while (t + 1 < s->n_types && i >= s->type_begin[t + 1]) ++t;
    return t;
}

static orc_px *raster_all(const orc_scene *s, double (*ecol)[3])
{
    orc_px *px = (orc_px *)malloc(sizeof(orc_px) * (size_t)(s->n > 0 ? s->n : 1));
    if (!px) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->n; ++i) {
        raster_one(s->x[i], s->y[i], s->z[i], s->h[i], s->m, s->p, s->W, s->H, s->rfac, s->rmin, &px[i]);
        if (ecol) {
            int t = type_of(s, i);
            if (s->vec && s->vec[t])
                colour_vector(&s->rgb[3 * i], s->beta[t], ecol[i]);
            else
                colour(s->It[i], s->cmap[t], s->cmap_len[t], s->beta[t], ecol[i]);
        }
    }
    return px;
}

static void fill_scene(orc_scene *s, int64_t n, const float *x, const float *y, const float *z,
                       const float *h, const double *It, int n_types, const int64_t *type_begin,
                       const float *const *cmap, const int *cmap_len, const double *beta,
                       const float m[12], const float p[5], int W, int H, float rfac, float rmin,
                       double sor, const double *rgb, const int *vec)
{
    s->rgb = rgb;
    s->vec = vec;
    s->n = n;
    s->x = x; s->y = y; s->z = z; s->h = h;
    s->It = It;
    s->n_types = n_types;
    s->type_begin = type_begin;
    s->cmap = cmap;
    s->cmap_len = cmap_len;
    s->beta = beta;
    memcpy(s->m, m, sizeof(s->m));
    memcpy(s->p, p, sizeof(s->p));
    s->W = W; s->H = H;
    s->rfac = rfac; s->rmin = rmin; s->sor = sor;
}

#define SCENE_ARGS                                                                                 \
    int64_t n, const float *x, const float *y, const float *z, const float *h, const double *It,   \
        int n_types, const int64_t *type_begin, const float *const *cmap, const int *cmap_len,     \
        const double *beta, const float m[12], const float p[5], int W, int H, float rfac,         \
        float rmin, double sor, const double *rgb, const int *vec
#define SCENE_PASS n, x, y, z, h, It, n_types, type_begin, cmap, cmap_len, beta, m, p, W, H, rfac, rmin, sor, rgb, vec

/* Per-particle raster outputs: X, Y, R, zc, e_r, e_g, e_b (FP64) and the active flag. */
int orc_raster(SCENE_ARGS, double *out7, int32_t *active, int32_t *box4)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    if (!px || !e) { free(px); free(e); return 2; }
    for (int64_t i = 0; i < n; ++i) {
        out7[0 * n + i] = px[i].X;
        out7[1 * n + i] = px[i].Y;
        out7[2 * n + i] = px[i].R;
        out7[3 * n + i] = px[i].zc;
        for (int c = 0; c < 3; ++c) out7[(4 + c) * n + i] = e[i][c];
        active[i] = px[i].active;
        if (box4) {
            box4[4 * i + 0] = px[i].i0;
            box4[4 * i + 1] = px[i].i1;
            box4[4 * i + 2] = px[i].j0;
            box4[4 * i + 3] = px[i].j1;
        }
    }
    free(px);
    free(e);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Direct render: the definition.  For each active particle (in index order) and each
 * covered pixel of its box, a[j][i][c] += e_c exp(-d^2 / sigma^2).  Rows are split among
 * threads; each pixel still sums its particles in index order, so the result does not
 * depend on the thread count.  a is H x W x 3, FP64.
 * ------------------------------------------------------------------------------------------ */
int orc_render(SCENE_ARGS, double *a)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    if (!px || !e) { free(px); free(e); return 2; }
    memset(a, 0, sizeof(double) * 3 * (size_t)W * (size_t)H);
    int nth = orc_num_threads();
    int band = (H + nth - 1) / nth;
#pragma omp parallel for schedule(static, 1)
    for (int b = 0; b < nth; ++b) {
        int r0 = b * band, r1 = r0 + band;
        if (r1 > H) r1 = H;
        for (int64_t k = 0; k < n; ++k) {
            const orc_px *o = &px[k];
            if (!o->active || o->j1 < r0 || o->j0 >= r1) continue;
            int ja = o->j0 > r0 ? o->j0 : r0, jb = o->j1 < r1 - 1 ? o->j1 : r1 - 1;
            for (int j = ja; j <= jb; ++j)
                for (int i = o->i0; i <= o->i1; ++i) {
                    if (!covered(o, i, j)) continue;
                    double w = weight(o, i, j, sor);
                    double *q = &a[3 * ((size_t)j * W + i)];
                    for (int c = 0; c < 3; ++c) q[c] += e[k][c] * w;
                }
        }
    }
    free(px);
    free(e);
    return ORC_OK;
}

/* Final transform (Section 2.1, radiative transfer along the line of sight with absorption
 * equal to emission): O = 1 - exp(-a) per channel, evaluated as -expm1(-a). */
void orc_final(int64_t count, const double *a, double *O)
{
    for (int64_t i = 0; i < count; ++i) O[i] = -expm1(-a[i]);
}

/* ------------------------------------------------------------------------------------------
 * Radiative transfer applied particle by particle (Section 2.1): for emission E and
 * absorption A the pixel value after one particle of weight w is
 *   I_out = I_in exp(-A w) + (E / A) (1 - exp(-A w)),
 * starting from black, particles in index order, per channel.  With A = E this must equal
 * the closed form of orc_final; it is written independently so each pins the other.
 * absorb_scale multiplies A relative to E (1 = the absorption-equals-emission mode).
 * ------------------------------------------------------------------------------------------ */
int orc_render_rt_sequential(SCENE_ARGS, double absorb_scale, double *I)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    if (!px || !e) { free(px); free(e); return 2; }
    memset(I, 0, sizeof(double) * 3 * (size_t)W * (size_t)H);
    for (int64_t k = 0; k < n; ++k) {
        const orc_px *o = &px[k];
        if (!o->active) continue;
        for (int j = o->j0; j <= o->j1; ++j)
            for (int i = o->i0; i <= o->i1; ++i) {
                if (!covered(o, i, j)) continue;
                double w = weight(o, i, j, sor);
                double *q = &I[3 * ((size_t)j * W + i)];
                for (int c = 0; c < 3; ++c) {
                    double E = e[k][c], A = absorb_scale * e[k][c];
                    if (A > 0.0) {
                        double t = exp(-A * w);
                        q[c] = q[c] * t + (E / A) * (1.0 - t);
                    } else {
                        q[c] = q[c] + E * w;
                    }
                }
            }
    }
    free(px);
    free(e);
    return ORC_OK;
}

/* Radiative transfer in depth order (Section 2.1: the image solves the transfer equation
 * along each line of sight; with absorption different from emission the result depends
 * on the order).  Absorption A = absorb[t] E for a particle of species t (absorb[t] >= 0).
 * The particles are applied from the farthest to the nearest (z_c descending, equal
 * depths by index), each to the pixels it covers, starting from a black background:
 *   I <- I exp(-A w) + (E / A)(1 - exp(-A w)),   I <- I + E w where A = 0.
 * I is H x W x 3, FP64.  With absorb[t] = 1 for every species this is 1 - exp(-a). */
static const orc_px *g_sort_px;
static int by_depth(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    float za = g_sort_px[a].zc, zb = g_sort_px[b].zc;
    if (za != zb) return za > zb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* The depth-ordered transfer at the pixels of a lattice only: (ox + stride a,
 * oy + stride b) for a, b >= 0 inside the image, written to L (ny x nx x 3, FP64,
 * nx = ceil((W - ox) / stride), ny likewise).  A pixel's value depends only on the
 * particles that cover it, so the particles whose box holds no lattice pixel are left out
 * before the depth sort; the rest are applied in the same order, so each lattice pixel
 * equals the full image's pixel exactly.  For checks of images too large to render whole. */
static int rt_depth_lattice(SCENE_ARGS, const double *absorb, int ox, int oy, int stride, double *L, double *Amap)
{
    if (stride < 1 || ox < 0 || oy < 0 || ox >= W || oy >= H) return 1;
    const int nx = (W - ox + stride - 1) / stride, ny = (H - oy + stride - 1) / stride;
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!px || !e || !ord) { free(px); free(e); free(ord); return 2; }
    int64_t na = 0;
    for (int64_t k = 0; k < n; ++k) {
        const orc_px *o = &px[k];
        if (!o->active) continue;
        /* first lattice column / row at or after the box's start */
        const int ia = o->i0 <= ox ? 0 : (o->i0 - ox + stride - 1) / stride;
        const int ja = o->j0 <= oy ? 0 : (o->j0 - oy + stride - 1) / stride;
        if (ox + ia * stride <= o->i1 && oy + ja * stride <= o->j1) ord[na++] = k;
    }
    g_sort_px = px;
    qsort(ord, (size_t)na, sizeof(int64_t), by_depth);
    memset(L, 0, sizeof(double) * 3 * (size_t)nx * (size_t)ny);
    if (Amap)
        for (size_t k = 0; k < 3 * (size_t)nx * (size_t)ny; ++k) Amap[k] = 1.0;
    for (int64_t q = 0; q < na; ++q) {
        const int64_t k = ord[q];
        const orc_px *o = &px[k];
        const double st = absorb[type_of(&s, k)];
        const int ia = o->i0 <= ox ? 0 : (o->i0 - ox + stride - 1) / stride;
        const int ja = o->j0 <= oy ? 0 : (o->j0 - oy + stride - 1) / stride;
        for (int b = ja; b < ny && oy + b * stride <= o->j1; ++b)
            for (int a = ia; a < nx && ox + a * stride <= o->i1; ++a) {
                const int i = ox + a * stride, j = oy + b * stride;
                if (!covered(o, i, j)) continue;
                double w = weight(o, i, j, sor);
                double *v = &L[3 * ((size_t)b * nx + a)];
                for (int c = 0; c < 3; ++c) {
                    double E = e[k][c], A = st * e[k][c];
                    if (A > 0.0) {
                        double t = exp(-A * w);
                        v[c] = v[c] * t + (E / A) * (1.0 - t);
                        if (Amap) Amap[3 * ((size_t)b * nx + a) + c] *= t;
                    } else {
                        v[c] = v[c] + E * w;
                    }
                }
            }
    }
    free(ord);
    free(px);
    free(e);
    return ORC_OK;
}

int orc_render_rt_depth_lattice(SCENE_ARGS, const double *absorb, int ox, int oy, int stride, double *L)
{
    return rt_depth_lattice(SCENE_PASS, absorb, ox, oy, stride, L, NULL);
}

/* The whole image: the lattice of stride 1. */
int orc_render_rt_depth(SCENE_ARGS, const double *absorb, double *I)
{
    if (W <= 0 || H <= 0) return ORC_OK;
    return rt_depth_lattice(SCENE_PASS, absorb, 0, 0, 1, I, NULL);
}

/* The same transfer as the affine map it applies to a pixel's incoming intensity:
 * I_out = alpha I_in + beta per channel, beta = the image above (black background) and
 * alpha = the product of exp(-A w) over the particles covering the pixel (1 where none
 * absorbs).  Maps of consecutive depth slabs compose far to near. */
int orc_render_rt_depth_map(SCENE_ARGS, const double *absorb, double *map_alpha, double *map_beta)
{
    if (W <= 0 || H <= 0) return ORC_OK;
    return rt_depth_lattice(SCENE_PASS, absorb, 0, 0, 1, map_beta, map_alpha);
}

/* Brute force: every pixel against every particle, no box and no tiles; coverage is the
 * bare FP32 test d2 < R2 on visible, finite particles. */
int orc_render_bruteforce(SCENE_ARGS, double *a)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    if (!px || !e) { free(px); free(e); return 2; }
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double *q = &a[3 * ((size_t)j * W + i)];
            q[0] = q[1] = q[2] = 0.0;
            for (int64_t k = 0; k < n; ++k) {
                const orc_px *o = &px[k];
                if (!(o->zc > p[3]) || !(o->zc <= p[4]) || !(isfinite(o->X) && isfinite(o->Y) && isfinite(o->R)))
                    continue;
                if (!covered(o, i, j)) continue;
                double w = weight(o, i, j, sor);
                for (int c = 0; c < 3; ++c) q[c] += e[k][c] * w;
            }
        }
    free(px);
    free(e);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Tile binning (Section 3.1 and the tile-list pseudocode and diagram of Section 3.2.1):
 * the image is cut into T x T tiles (the last column / row of tiles may be partial); a
 * particle joins tile (tx, ty) when the distance from its centre to the tile centre is
 * below 0.75 radius + sqrt(2) T / 2.  The radius here is the clamped one, R / 0.75, so the
 * 0.75 radius term is the support R.  Candidate tiles are those meeting the pixel box.
 * FP32, each operation rounded once:
 *   cx = (tx + 0.5) T, cy = (ty + 0.5) T  (full nominal tile, also for partial tiles)
 *   ex = cx - X, ey = cy - Y, q = ex ex + ey ey
 *   thr = R + 0.70710677 T (product rounded first), member iff q < thr thr.
 * Lists come out in ascending particle index.  counts[n_tiles]; offsets[n_tiles + 1];
 * members may be NULL (counts only); returns the total number of pairs in *total.
 * ------------------------------------------------------------------------------------------ */
static int tile_member(const orc_px *o, int tx, int ty, int T)
{
    float hd = 0.70710677f * (float)T;
    float cx = ((float)tx + 0.5f) * (float)T;
    float cy = ((float)ty + 0.5f) * (float)T;
    float ex = cx - o->X, ey = cy - o->Y;
    float q = ex * ex + ey * ey;
    float thr = o->R + hd;
    return q < thr * thr;
}

int orc_bin(SCENE_ARGS, int T, int32_t *counts, int64_t *offsets, int32_t *members,
            int64_t capacity, int64_t *total)
{
    if (T < 1) return ORC_EINVAL;
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    orc_px *px = raster_all(&s, NULL);
    if (!px) return 2;
    int ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    int64_t nt = (int64_t)ntx * nty;
    memset(counts, 0, sizeof(int32_t) * (size_t)nt);
    for (int64_t k = 0; k < n; ++k) {
        const orc_px *o = &px[k];
        if (!o->active) continue;
        for (int ty = o->j0 / T; ty <= o->j1 / T; ++ty)
            for (int tx = o->i0 / T; tx <= o->i1 / T; ++tx)
                if (tile_member(o, tx, ty, T)) counts[(int64_t)ty * ntx + tx]++;
    }
    offsets[0] = 0;
    for (int64_t t = 0; t < nt; ++t) offsets[t + 1] = offsets[t] + counts[t];
    *total = offsets[nt];
    if (members) {
        if (*total > capacity) { free(px); return 3; }
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
        if (!cur) { free(px); return 2; }
        memcpy(cur, offsets, sizeof(int64_t) * (size_t)nt);
        for (int64_t k = 0; k < n; ++k) {
            const orc_px *o = &px[k];
            if (!o->active) continue;
            for (int ty = o->j0 / T; ty <= o->j1 / T; ++ty)
                for (int tx = o->i0 / T; tx <= o->i1 / T; ++tx)
                    if (tile_member(o, tx, ty, T)) members[cur[(int64_t)ty * ntx + tx]++] = (int32_t)k;
        }
        free(cur);
    }
    free(px);
    return ORC_OK;
}

/* Work of one frame, in the units the splat and binning costs are counted in:
 * out[0] = active particles, out[1] = covered (particle, pixel) pairs, i.e. kernel
 * evaluations the definition of Section 2.1 makes (every pixel whose centre lies inside a
 * particle's support gets one), out[2] = (particle, tile) pairs under the tile rule of
 * Section 3.2.1 with edge T (0 skips it). */
int orc_count_work(SCENE_ARGS, int T, int64_t *out)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    orc_px *px = raster_all(&s, NULL);
    if (!px) return 2;
    int64_t act = 0, cov = 0, tp = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : act, cov, tp)
    for (int64_t k = 0; k < n; ++k) {
        const orc_px *o = &px[k];
        if (!o->active) continue;
        ++act;
        for (int j = o->j0; j <= o->j1; ++j)
            for (int i = o->i0; i <= o->i1; ++i) cov += covered(o, i, j);
        if (T > 0)
            for (int ty = o->j0 / T; ty <= o->j1 / T; ++ty)
                for (int tx = o->i0 / T; tx <= o->i1 / T; ++tx) tp += tile_member(o, tx, ty, T);
    }
    out[0] = act;
    out[1] = cov;
    out[2] = tp;
    free(px);
    return ORC_OK;
}

/* Tiled render (Section 3.1: each tile renders its own particle list, pixels stay local to
 * the tile): for every tile, its members in list order, the covered pixels of the tile. */
int orc_render_tiled(SCENE_ARGS, int T, double *a)
{
    if (T < 1) return ORC_EINVAL;
    int ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    int64_t nt = (int64_t)ntx * nty;
    int32_t *counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt + 1));
    int64_t total = 0;
    if (!counts || !offs) { free(counts); free(offs); return 2; }
    int rc = orc_bin(SCENE_PASS, T, counts, offs, NULL, 0, &total);
    if (rc) { free(counts); free(offs); return rc; }
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!mem) { free(counts); free(offs); return 2; }
    rc = orc_bin(SCENE_PASS, T, counts, offs, mem, total, &total);
    if (rc) { free(counts); free(offs); free(mem); return rc; }
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    double (*e)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_px *px = raster_all(&s, e);
    if (!px || !e) { free(px); free(e); free(counts); free(offs); free(mem); return 2; }
    memset(a, 0, sizeof(double) * 3 * (size_t)W * (size_t)H);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nt; ++t) {
        int tx = (int)(t % ntx), ty = (int)(t / ntx);
        int x0 = tx * T, y0 = ty * T;
        int x1 = x0 + T - 1 < W - 1 ? x0 + T - 1 : W - 1;
        int y1 = y0 + T - 1 < H - 1 ? y0 + T - 1 : H - 1;
        for (int64_t q = offs[t]; q < offs[t + 1]; ++q) {
            int32_t k = mem[q];
            const orc_px *o = &px[k];
            for (int j = y0; j <= y1; ++j) {
                if (j < o->j0 || j > o->j1) continue;
                for (int i = x0; i <= x1; ++i) {
                    if (i < o->i0 || i > o->i1 || !covered(o, i, j)) continue;
                    double w = weight(o, i, j, sor);
                    double *pa = &a[3 * ((size_t)j * W + i)];
                    for (int c = 0; c < 3; ++c) pa[c] += e[k][c] * w;
                }
            }
        }
    }
    free(px);
    free(e);
    free(counts);
    free(offs);
    free(mem);
    return ORC_OK;
}

/* Pixels covered by particle k: writes (i, j) pairs, returns their number (for the
 * conservativeness check of the binning rule). */
int64_t orc_covered_pixels(SCENE_ARGS, int64_t k, int32_t *ij, int64_t capacity)
{
    orc_scene s;
    fill_scene(&s, SCENE_PASS);
    orc_px o;
    raster_one(x[k], y[k], z[k], h[k], s.m, s.p, W, H, rfac, rmin, &o);
    if (!o.active) return 0;
    int64_t cnt = 0;
    for (int j = o.j0; j <= o.j1; ++j)
        for (int i = o.i0; i <= o.i1; ++i)
            if (covered(&o, i, j)) {
                if (cnt < capacity) {
                    ij[2 * cnt] = i;
                    ij[2 * cnt + 1] = j;
                }
                ++cnt;
            }
    return cnt;
}
