/*
 * oracle.c -- plain, slow, obviously correct CPU reference of the bricked
 * multi-resolution raycaster.  TEST INFRASTRUCTURE ONLY: tests, the package's
 * smoke check and the benchmark's CPU-baseline leg call it; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * What it computes, and the passages it follows (Drees & Risse, "Palace",
 * arXiv 2509.26213):
 *   - chunk addressing h = floor(g / C), l = g mod C            (Sec. III-A)
 *   - LOD pyramid: level 0 full resolution, coarser levels by smoothing and
 *     downsampling, uniform physical size so spacing grows      (Sec. III-D)
 *   - one page directory per level, indexed by level            (Sec. III-E)
 *   - dynamic LOD selection while rendering                    (Sec. V-C; App.)
 *   - front-to-back emission/absorption compositing (DVR) with a 1D RGBA
 *     transfer function                                         (Sec. IV-A; Fig. 1)
 *   - maximum-opacity projection (MOP), and maximum-intensity projection
 *     beside it                                                 (Sec. V-A; Table I)
 *   - progressive preview: absent bricks replaced by coarser
 *     resident levels                                           (Sec. III-H)
 * The paper gives no formulas for ray setup, interpolation, LOD choice or
 * compositing; the readings used here are listed in the design notes and in
 * the comments of each function.
 *
 * Two layers:
 *   decision layer -- IEEE binary32, round to nearest, no contraction
 *     (compile with -ffp-contract=off), operations in the written order:
 *     pixel -> ray, slab entry/exit, sample positions, LOD level, voxel index,
 *     brick id and local position.  These decide integers, so both sides must
 *     take them in the same precision.
 *   value layer -- float64: decoded voxel values, trilinear interpolation,
 *     transfer-function lookup, compositing, adjoint.
 *
 * Dense volume layout everywhere: x fastest (index x + Dx*(y + Dy*z)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LEVELS 16

enum { ORC_U8 = 0, ORC_U16 = 1, ORC_F16 = 2, ORC_F32 = 3 };

typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float tan_half_fov; /* tan of half the vertical field of view */
    float aspect;       /* w / h */
    int32_t w, h;
} orc_camera;

typedef struct {
    float step;         /* sample spacing dt, level-0 voxel units */
    float et;           /* early termination: stop after a sample once 1 - T >= et */
    float bg[4];        /* background RGBA behind the volume */
    int32_t lod_mode;   /* 0: every sample on level 0; 1: footprint LOD */
    int32_t lod_bias;   /* added to the footprint level before clamping */
    int32_t level_step; /* 1: sample spacing and opacity scaled with the level (below) */
} orc_params;

typedef struct {
    int32_t nlevels;
    int32_t dtype;                       /* ORC_U8 .. ORC_F32 */
    int32_t brick;                       /* brick edge B, for reporting ids */
    int64_t dims[ORC_MAX_LEVELS][3];     /* dims per level */
    const void *data[ORC_MAX_LEVELS];    /* dense voxels per level */
} orc_volume;

/* ------------------------------------------------------------ levels */

/* Sec. III-D: dims shrink level by level; here D_{l+1} = ceil(D_l / 2). */
void orc_level_dims(const int64_t D0[3], int nlevels, int64_t *out /* [nlevels][3] */)
{
    for (int a = 0; a < 3; ++a) out[a] = D0[a];
    for (int l = 1; l < nlevels; ++l)
        for (int a = 0; a < 3; ++a) out[3 * l + a] = (out[3 * (l - 1) + a] + 1) / 2;
}

/* ------------------------------------------------- half precision */

/* binary16 -> double, exact (IEEE 754 binary16 definition). */
double orc_half_to_double(uint16_t h)
{
    int s = h >> 15, e = (h >> 10) & 0x1f, m = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(m | 0x400), e - 25);
    return s ? -v : v;
}

/* binary32 -> binary16, round to nearest even (IEEE 754), via exact double
 * arithmetic: pick the nearest representable half, ties to even mantissa. */
uint16_t orc_float_to_half(float f)
{
    double x = (double)f;
    uint16_t sign = signbit(x) ? 0x8000 : 0;
    double a = fabs(x);
    if (isnan(x)) return sign | 0x7e00;
    if (a >= 65520.0) return sign | 0x7c00; /* rounds to infinity */
    /* quantum of the binade containing a (subnormal quantum 2^-24) */
    int e;
    if (a < ldexp(1.0, -14)) {
        e = -24;
    } else {
        int ex;
        frexp(a, &ex);  /* a = m * 2^ex, m in [0.5, 1) */
        e = ex - 11;    /* 10 mantissa bits after the leading one */
    }
    double q = ldexp(1.0, e);
    double n = floor(a / q);       /* exact: a/q is a power-of-two scaling */
    double r = a - n * q;          /* exact remainder */
    if (r > q / 2 || (r == q / 2 && fmod(n, 2.0) != 0.0)) n += 1.0;
    double v = n * q;
    /* encode v */
    if (v == 0.0) return sign;
    if (v < ldexp(1.0, -14)) return sign | (uint16_t)(v / ldexp(1.0, -24));
    int ex;
    double m = frexp(v, &ex); /* v = m 2^ex, m in [0.5,1) */
    int E = ex - 1 + 15;
    if (E >= 31) return sign | 0x7c00;
    uint16_t mant = (uint16_t)((m * 2.0 - 1.0) * 1024.0);
    return sign | (uint16_t)(E << 10) | mant;
}

/* Reduced-precision storage: a uint16 voxel u stored as binary16 of the
 * binary32 quotient u / 65535 (one correctly rounded float division, then
 * round to nearest even). */
void orc_u16_to_f16(int64_t n, const uint16_t *src, uint16_t *dst)
{
    /* all 65536 inputs converted once, then looked up */
    uint16_t *tab = malloc(sizeof(uint16_t) * 65536);
    for (int u = 0; u < 65536; ++u) tab[u] = orc_float_to_half((float)u / 65535.0f);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) dst[i] = tab[src[i]];
    free(tab);
}

/* u8 -> float32 normalised value (the normalisation u / 255 of the storage
 * convention, rounded once to binary32: one correctly rounded float division). */
void orc_u8_to_f32(int64_t n, const uint8_t *src, float *dst)
{
    for (int64_t i = 0; i < n; ++i) dst[i] = (float)src[i] / 255.0f;
}

/* u16 -> float32 normalised value (u / 65535, rounded once to binary32). */
void orc_u16_to_f32(int64_t n, const uint16_t *src, float *dst)
{
    for (int64_t i = 0; i < n; ++i) dst[i] = (float)src[i] / 65535.0f;
}

/* ------------------------------------------------------ downsample */

/*
 * Sec. III-D: level l+1 from level l by a 2x2x2 box filter (the paper
 * smooths, then halves the resolution).  Coarse voxel i averages children 2i and 2i+1 per axis;
 * a child index beyond the fine edge is replaced by the last fine voxel.
 *   u8/u16: integer mean rounded half up, (sum + 4) >> 3
 *   f16/f32: binary32 sum of the eight children in the order
 *            (dz, dy, dx) = (0,0,0),(0,0,1),(0,1,0),(0,1,1),(1,0,0),...,
 *            times 0.125, then (f16) rounded to nearest even.
 */
int orc_downsample(int dtype, const int64_t D[3], const void *src, void *dst)
{
    int64_t Dn[3];
    for (int a = 0; a < 3; ++a) Dn[a] = (D[a] + 1) / 2;
    if (dtype < ORC_U8 || dtype > ORC_F32) return -1;
    /* binary16 decode table (every value through orc_half_to_double) */
    float *half_tab = NULL;
    if (dtype == ORC_F16) {
        half_tab = malloc(sizeof(float) * 65536);
        if (!half_tab) return -2;
        for (int h = 0; h < 65536; ++h) half_tab[h] = (float)orc_half_to_double((uint16_t)h);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t z = 0; z < Dn[2]; ++z)
        for (int64_t y = 0; y < Dn[1]; ++y)
            for (int64_t x = 0; x < Dn[0]; ++x) {
                int64_t isum = 0;
                float fsum = 0.0f;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            int64_t cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                            if (cx > D[0] - 1) cx = D[0] - 1;
                            if (cy > D[1] - 1) cy = D[1] - 1;
                            if (cz > D[2] - 1) cz = D[2] - 1;
                            int64_t ci = cx + D[0] * (cy + D[1] * cz);
                            switch (dtype) {
                            case ORC_U8: isum += ((const uint8_t *)src)[ci]; break;
                            case ORC_U16: isum += ((const uint16_t *)src)[ci]; break;
                            case ORC_F16: fsum = fsum + half_tab[((const uint16_t *)src)[ci]]; break;
                            case ORC_F32: fsum = fsum + ((const float *)src)[ci]; break;
                            }
                        }
                int64_t o = x + Dn[0] * (y + Dn[1] * z);
                switch (dtype) {
                case ORC_U8: ((uint8_t *)dst)[o] = (uint8_t)((isum + 4) >> 3); break;
                case ORC_U16: ((uint16_t *)dst)[o] = (uint16_t)((isum + 4) >> 3); break;
                case ORC_F16: ((uint16_t *)dst)[o] = orc_float_to_half(fsum * 0.125f); break;
                case ORC_F32: ((float *)dst)[o] = fsum * 0.125f; break;
                }
            }
    free(half_tab);
    return 0;
}

/* ------------------------------------------------- decision layer */

typedef struct {
    float o[3], d[3];
    float t0, t1;
    int hit;
} orc_ray;

/*
 * Pixel (px, py) -> ray (decision layer, binary32).  Pixel centres at +0.5;
 * normalised device coordinates u in (-1,1) left to right, v in (-1,1)
 * bottom to top (image rows run downward).  Direction
 *   d = fwd + (u * tan * aspect) * right + (v * tan) * up, then d / sqrt(|d|^2).
 * Entry/exit (Fig. 1's entry_exit_points): slab test against the box
 * [0, D0) in level-0 voxel units, entry clamped at t = 0 when the eye is
 * inside.  The ray hits when t0 < t1.
 */
void orc_make_ray(const orc_camera *c, const int64_t D0[3], int32_t px, int32_t py, orc_ray *r)
{
    float u = (((float)px + 0.5f) / (float)c->w) * 2.0f - 1.0f;
    float v = 1.0f - (((float)py + 0.5f) / (float)c->h) * 2.0f;
    float tx = c->tan_half_fov * c->aspect;
    float cx = u * tx;
    float cy = v * c->tan_half_fov;
    float dd[3];
    for (int a = 0; a < 3; ++a) dd[a] = (c->fwd[a] + cx * c->right[a]) + cy * c->up[a];
    float len2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2];
    float inv = 1.0f / sqrtf(len2);
    for (int a = 0; a < 3; ++a) {
        r->d[a] = dd[a] * inv;
        r->o[a] = c->eye[a];
    }
    float t0 = 0.0f, t1 = INFINITY;
    int hit = 1;
    for (int a = 0; a < 3; ++a) {
        float Da = (float)D0[a];
        if (r->d[a] == 0.0f) {
            if (r->o[a] < 0.0f || r->o[a] >= Da) hit = 0;
            continue;
        }
        float ta = (0.0f - r->o[a]) / r->d[a];
        float tb = (Da - r->o[a]) / r->d[a];
        float tn = ta < tb ? ta : tb;
        float tf = ta < tb ? tb : ta;
        if (tn > t0) t0 = tn;
        if (tf < t1) t1 = tf;
    }
    r->t0 = t0;
    r->t1 = t1;
    r->hit = hit && (t0 < t1);
}

/* Sample k sits at t_k = t0 + k * dt (binary32 product, then sum) and exists
 * while t_k < t1; no jitter and no half-step offset. */
static inline float sample_t(const orc_ray *r, float dt, int64_t k)
{
    return r->t0 + (float)k * dt;
}

/*
 * Level-scaled sampling (an extension: the paper fixes no step rule for coarse levels, Sec.
 * V-C): a sample on level l stands for 2^l reference steps, so
 *   t_0 = t0,  t_{k+1} = t_k + dt * 2^{l_k}   (binary32 sum; the scaling is exact),
 * and its opacity is corrected to the longer step: a' = 1 - (1 - a)^(2^l).
 */
static inline float next_t_level_step(float t, float dt, int level)
{
    return t + ldexpf(dt, level);
}

/* Footprint scale: world size of one pixel at unit distance, in level-0
 * voxels: (2 * tan_half_fov) / h. */
static inline float lod_scale(const orc_camera *c)
{
    return (2.0f * c->tan_half_fov) / (float)c->h;
}

/*
 * Dynamic LOD (Sec. V-C, Appendix; no formula given).  Reading: the pixel
 * footprint at depth t is q = t * lod_scale level-0 voxels; use the level
 * whose voxel size 2^l is the largest power of two not above q (plus a bias):
 *   l = clamp(ilogb(q) + bias, 0, L - 1), and l = 0 when q has no normal
 *   exponent (q = 0 or subnormal).
 */
static inline int lod_level(float t, float scale, int bias, int nlevels, int mode)
{
    if (!mode) return 0;
    float q = t * scale;
    int e;
    if (!(q >= 0x1.0p-126f))
        e = -127;
    else
        e = ilogbf(q);
    int l = e + bias;
    if (l < 0) l = 0;
    if (l > nlevels - 1) l = nlevels - 1;
    return l;
}

typedef struct {
    int level;
    int64_t i0[3];   /* clamped lower corner voxel on the level grid */
    float w[3];      /* interpolation weights (0 on clamped axes) */
    int64_t brick[3];
    int64_t local[3];
    int64_t brick_id;
} orc_resolve;

/*
 * Position p (level-0 units) on level l.  Voxel centres at i + 0.5, spacing
 * s_l = D0 / D_l per axis (uniform physical size, Sec. III-D), so the grid
 * coordinate is x = p * (D_l / D0) - 0.5, with the ratio rounded once.
 * Clamp to edge: i = floor(x); i < 0 -> i0 = 0, weight 0; i >= D_l - 1 ->
 * i0 = D_l - 1, weight 0; else i0 = i, weight x - floor(x).
 * Chunk addressing (Sec. III-A): brick h = i0 div B, local l = i0 mod B,
 * brick id = hx + nbx * (hy + nby * hz), nb = ceil(D_l / B).
 */
static void resolve(const orc_volume *V, int level, const float p[3], orc_resolve *R)
{
    const int64_t *D0 = V->dims[0], *Dl = V->dims[level];
    int64_t nb[3];
    R->level = level;
    for (int a = 0; a < 3; ++a) {
        float ratio = (float)Dl[a] / (float)D0[a];
        float x = p[a] * ratio - 0.5f;
        float fx = floorf(x);
        int64_t i = (int64_t)fx;
        if (i < 0) {
            R->i0[a] = 0;
            R->w[a] = 0.0f;
        } else if (i >= Dl[a] - 1) {
            R->i0[a] = Dl[a] - 1;
            R->w[a] = 0.0f;
        } else {
            R->i0[a] = i;
            R->w[a] = x - fx;
        }
        R->brick[a] = R->i0[a] / V->brick;
        R->local[a] = R->i0[a] % V->brick;
        nb[a] = (Dl[a] + V->brick - 1) / V->brick;
    }
    R->brick_id = R->brick[0] + nb[0] * (R->brick[1] + nb[1] * R->brick[2]);
}

/* --------------------------------------------------- value layer */

/* Normalised voxel value: u8 / 255, u16 / 65535, floats as stored. */
static inline double voxel(const orc_volume *V, int level, int64_t x, int64_t y, int64_t z)
{
    const int64_t *D = V->dims[level];
    int64_t i = x + D[0] * (y + D[1] * z);
    switch (V->dtype) {
    case ORC_U8: return (double)((const uint8_t *)V->data[level])[i] / 255.0;
    case ORC_U16: return (double)((const uint16_t *)V->data[level])[i] / 65535.0;
    case ORC_F16: return orc_half_to_double(((const uint16_t *)V->data[level])[i]);
    default: return (double)((const float *)V->data[level])[i];
    }
}

typedef struct {
    double v;            /* trilinear value (before clamp) */
    int64_t corner[8];   /* dense indices of the 8 corners on the level */
    double cw[8];        /* their trilinear weights */
} orc_interp;

/* Trilinear interpolation on the level grid (the global grid: no bricks). */
static void interp(const orc_volume *V, const orc_resolve *R, orc_interp *I)
{
    const int64_t *D = V->dims[R->level];
    int64_t i1[3];
    for (int a = 0; a < 3; ++a) i1[a] = R->i0[a] + 1 < D[a] ? R->i0[a] + 1 : D[a] - 1;
    double wx = R->w[0], wy = R->w[1], wz = R->w[2];
    double v = 0.0;
    int c = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx, ++c) {
                int64_t x = dx ? i1[0] : R->i0[0];
                int64_t y = dy ? i1[1] : R->i0[1];
                int64_t z = dz ? i1[2] : R->i0[2];
                double w = (dx ? wx : 1.0 - wx) * (dy ? wy : 1.0 - wy) * (dz ? wz : 1.0 - wz);
                I->corner[c] = x + D[0] * (y + D[1] * z);
                I->cw[c] = w;
                v += w * voxel(V, R->level, x, y, z);
            }
    I->v = v;
}

typedef struct {
    double rgba[4];
    double x;       /* TF coordinate */
    int i;          /* lower TF entry */
    double w;       /* weight of entry i + 1 */
    int inside;     /* value was inside [0, 1] (clamp inactive) */
} orc_tflookup;

/* The TF at coordinate x in [0, 255]: i = min(floor(x), 254),
 * rgba = tf[i] + (x - i) * (tf[i+1] - tf[i]). */
static void tf_at(const float *tf, double x, orc_tflookup *L)
{
    L->x = x;
    int i = (int)floor(x);
    if (i > 254) i = 254;
    double w = x - (double)i;
    L->i = i;
    L->w = w;
    for (int ch = 0; ch < 4; ++ch) {
        double a = tf[4 * i + ch], b = tf[4 * (i + 1) + ch];
        L->rgba[ch] = a + w * (b - a);
    }
}

/* 1D RGBA transfer function with N = 256 entries (Fig. 1's grey_ramp_tf is
 * such a table): value clamped to [0, 1], x = v * (N - 1), then tf_at(x). */
static void tf_lookup(const float *tf, double v, orc_tflookup *L)
{
    L->inside = (v >= 0.0 && v <= 1.0);
    double vc = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    tf_at(tf, vc * 255.0, L);
}

/* --------------------------------------------------------- tracing */

typedef struct {
    int32_t k;
    uint32_t t_bits;
    int32_t level;
    int32_t i0[3];
    int32_t local[3];
    int64_t brick_id;
} orc_trace_rec;

/* Decision-layer records of the first max_samples samples of pixel (px,py)
 * (no early termination: every sample up to the exit).  Returns the number of
 * samples of the ray (may exceed max_samples). */
int64_t orc_trace(const orc_volume *V, const orc_camera *c, const orc_params *P, int32_t px,
                  int32_t py, int64_t max_samples, orc_trace_rec *out)
{
    orc_ray r;
    orc_make_ray(c, V->dims[0], px, py, &r);
    if (!r.hit) return 0;
    float scale = lod_scale(c);
    int64_t k = 0;
    float t = r.t0;
    int l = 0;
    for (;; ++k) {
        t = P->level_step ? (k ? next_t_level_step(t, P->step, l) : r.t0) : sample_t(&r, P->step, k);
        if (!(t < r.t1)) break;
        l = lod_level(t, scale, P->lod_bias, V->nlevels, P->lod_mode);
        if (k >= max_samples) continue;
        float p[3];
        for (int a = 0; a < 3; ++a) p[a] = r.o[a] + t * r.d[a];
        orc_resolve R;
        resolve(V, l, p, &R);
        orc_trace_rec *q = &out[k];
        q->k = (int32_t)k;
        memcpy(&q->t_bits, &t, 4);
        q->level = l;
        for (int a = 0; a < 3; ++a) {
            q->i0[a] = (int32_t)R.i0[a];
            q->local[a] = (int32_t)R.local[a];
        }
        q->brick_id = R.brick_id;
    }
    return k;
}

/* ---------------------------------------------------------- render */

/*
 * Front-to-back emission/absorption (DVR, Sec. IV-A), no opacity correction:
 * for k = 0, 1, ...:  C += T * alpha_k * rgb_k;  T *= (1 - alpha_k);
 * stop after sample k once 1 - T >= et.  Output rgb = C + T * bg_rgb,
 * a = (1 - T) + T * bg_a.
 *
 * Early termination compares a float64 T here and a float32 T on the GPU; the
 * two may decide differently when 1 - T lands within rounding of et.  Both
 * outcomes are correct, so the oracle reports the first sample whose margin
 * |1 - T - et| is below `amb` and, as the alternate, the result with that one
 * decision flipped.
 *
 * flip_k >= 0 flips the termination decision at sample flip_k.
 * Returns n (samples composited); *amb_k receives the first ambiguous sample
 * or -1.
 */
typedef struct {
    double C[3], T;
} orc_state;

/* Page-table index of (level, brick id): the levels' tables laid end to end, level 0
 * first, each with ceil(D_l / B) bricks per axis (Sec. III-E). */
static int64_t pt_index(const orc_volume *V, int level, int64_t brick_id)
{
    int64_t off = 0;
    for (int l = 0; l < level; ++l) {
        int64_t n = 1;
        for (int a = 0; a < 3; ++a) n *= (V->dims[l][a] + V->brick - 1) / V->brick;
        off += n;
    }
    return off + brick_id;
}

/*
 * Progressive preview (Sec. III-H, Rendering: a low-resolution image from coarser LOD levels
 * first, refined as bricks arrive).  Reading: with a residency map (one byte per page-table
 * index), a sample whose brick on its level l is not resident is taken on the finest coarser
 * level l' > l whose brick at the same position is resident; when none is, the sample
 * composites nothing.  Returns 0 when the sample is skipped, else 1 with R resolved on the
 * level used.
 */
static int resolve_resident(const orc_volume *V, int level, const float p[3], const uint8_t *resident,
                            orc_resolve *R)
{
    resolve(V, level, p, R);
    if (!resident || resident[pt_index(V, level, R->brick_id)]) return 1;
    for (int l = level + 1; l < V->nlevels; ++l) {
        resolve(V, l, p, R);
        if (resident[pt_index(V, l, R->brick_id)]) return 1;
    }
    return 0;
}

static int64_t march(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
                     const uint8_t *resident, const orc_ray *r, int64_t flip_k, double amb, int64_t *amb_k,
                     orc_state *S)
{
    float scale = lod_scale(c);
    S->C[0] = S->C[1] = S->C[2] = 0.0;
    S->T = 1.0;
    if (amb_k) *amb_k = -1;
    if (!r->hit) return 0;
    int64_t k = 0;
    float t = r->t0;
    int l = 0;
    for (;; ++k) {
        t = P->level_step ? (k ? next_t_level_step(t, P->step, l) : r->t0) : sample_t(r, P->step, k);
        if (!(t < r->t1)) break;
        float p[3];
        for (int a = 0; a < 3; ++a) p[a] = r->o[a] + t * r->d[a];
        l = lod_level(t, scale, P->lod_bias, V->nlevels, P->lod_mode);
        orc_resolve R;
        if (!resolve_resident(V, l, p, resident, &R)) continue; /* preview: nothing resident here */
        orc_interp I;
        interp(V, &R, &I);
        orc_tflookup L;
        tf_lookup(tf, I.v, &L);
        double al = L.rgba[3];
        if (P->level_step && l > 0) {
            double om = 1.0 - al; /* (1 - a)^(2^l) by l squarings */
            for (int q = 0; q < l; ++q) om *= om;
            al = 1.0 - om;
        }
        for (int ch = 0; ch < 3; ++ch) S->C[ch] += S->T * al * L.rgba[ch];
        S->T *= (1.0 - al);
        double margin = (1.0 - S->T) - (double)P->et;
        int stop = margin >= 0.0;
        if (amb_k && *amb_k < 0 && fabs(margin) < amb) *amb_k = k;
        if (k == flip_k) stop = !stop;
        if (stop) {
            ++k;
            break;
        }
    }
    return k;
}

static void finish(const orc_state *S, const orc_params *P, double *rgba)
{
    for (int ch = 0; ch < 3; ++ch) rgba[ch] = S->C[ch] + S->T * (double)P->bg[ch];
    rgba[3] = (1.0 - S->T) + S->T * (double)P->bg[3];
}

/*
 * Render npix pixels (pix = [npix][2] px,py; NULL = all pixels row-major).
 * out_rgba [npix][4], out_n [npix]; alt_rgba / alt_n receive the alternate
 * (flipped early-termination) result where amb_flag[i] = 1, else a copy.
 */
static int render_impl(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
                       const uint8_t *resident, const int32_t *pix, int64_t npix, double amb, double *out_rgba,
                       int32_t *out_n, double *alt_rgba, int32_t *alt_n, int32_t *amb_flag, int nthreads)
{
    if (V->nlevels < 1 || V->nlevels > ORC_MAX_LEVELS || V->brick < 1) return -1;
    if (!pix) npix = (int64_t)c->w * c->h;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < npix; ++i) {
        int32_t px = pix ? pix[2 * i] : (int32_t)(i % c->w);
        int32_t py = pix ? pix[2 * i + 1] : (int32_t)(i / c->w);
        orc_ray r;
        orc_make_ray(c, V->dims[0], px, py, &r);
        orc_state S;
        int64_t ak;
        int64_t n = march(V, c, tf, P, resident, &r, -1, amb, &ak, &S);
        finish(&S, P, &out_rgba[4 * i]);
        out_n[i] = (int32_t)n;
        if (alt_rgba) {
            if (ak >= 0) {
                orc_state S2;
                int64_t n2 = march(V, c, tf, P, resident, &r, ak, amb, NULL, &S2);
                finish(&S2, P, &alt_rgba[4 * i]);
                alt_n[i] = (int32_t)n2;
                amb_flag[i] = 1;
            } else {
                memcpy(&alt_rgba[4 * i], &out_rgba[4 * i], 4 * sizeof(double));
                alt_n[i] = (int32_t)n;
                amb_flag[i] = 0;
            }
        }
    }
    return 0;
}

int orc_render(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
               const int32_t *pix, int64_t npix, double amb, double *out_rgba, int32_t *out_n,
               double *alt_rgba, int32_t *alt_n, int32_t *amb_flag, int nthreads)
{
    return render_impl(V, c, tf, P, NULL, pix, npix, amb, out_rgba, out_n, alt_rgba, alt_n, amb_flag, nthreads);
}

/* orc_render with a residency map (one byte per page-table index, levels end to end): the
 * progressive preview of resolve_resident.  out_n counts every sample the ray passed,
 * skipped ones included. */
int orc_render_preview(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
                       const uint8_t *resident, const int32_t *pix, int64_t npix, double amb, double *out_rgba,
                       int32_t *out_n, double *alt_rgba, int32_t *alt_n, int32_t *amb_flag, int nthreads)
{
    if (!resident) return -1;
    return render_impl(V, c, tf, P, resident, pix, npix, amb, out_rgba, out_n, alt_rgba, alt_n, amb_flag, nthreads);
}

/* ----------------------------------------------- maximum projections */

/*
 * Maximum-opacity projection (MOP; the Kidney renderings of Sec. V-A, Table I)
 * and maximum-intensity projection (MIP).  The paper names MOP without a
 * formula; the reading used here visits every sample of the ray (no early
 * termination) and keeps one of them:
 *   MOP -- the first sample of largest TF opacity alpha_k (a later sample
 *          replaces it only when its opacity is strictly larger), with its
 *          TF colour c_k;
 *   MIP -- the largest TF coordinate x_k = 255 clamp(v_k, 0, 1), then the TF
 *          at that coordinate gives (c, alpha);
 * and composites the kept (c, alpha) once over the background:
 *   rgb = alpha c + (1 - alpha) bg_rgb,   a = alpha + (1 - alpha) bg_a.
 * A ray that misses the box gives bg, and so does MOP when every opacity is 0.
 */
enum { ORC_MOP = 1, ORC_MIP = 2 };

static void composite_one(const double rgba[4], const orc_params *P, double *out)
{
    double al = rgba[3];
    for (int ch = 0; ch < 3; ++ch) out[ch] = al * rgba[ch] + (1.0 - al) * (double)P->bg[ch];
    out[3] = al + (1.0 - al) * (double)P->bg[3];
}

/* TF lookup of sample k of ray r (value layer); returns 0 past the exit, 2 for a sample that
 * a preview's residency map leaves out (nothing resident at its position). */
static int sample_lookup(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
                         const uint8_t *resident, const orc_ray *r, int64_t k, orc_tflookup *L)
{
    float t = sample_t(r, P->step, k);
    if (!(t < r->t1)) return 0;
    float p[3];
    for (int a = 0; a < 3; ++a) p[a] = r->o[a] + t * r->d[a];
    int l = lod_level(t, lod_scale(c), P->lod_bias, V->nlevels, P->lod_mode);
    orc_resolve R;
    if (!resolve_resident(V, l, p, resident, &R)) return 2;
    orc_interp I;
    interp(V, &R, &I);
    tf_lookup(tf, I.v, L);
    return 1;
}

/*
 * Render npix pixels in projection mode `mode` (ORC_MOP or ORC_MIP); pixel
 * list as in orc_render.  out_n receives the samples of the ray.
 * MOP compares float64 opacities here and float32 ones on the GPU, so any
 * sample whose opacity lies within `amb` of the maximum may be the one kept:
 * lo and hi receive, per channel, the least and greatest output over those
 * samples (both equal out when no other sample is that close).  MIP's output
 * is continuous in the maximum, so there lo = hi = out.
 */
int orc_render_max(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P, int mode,
                   const uint8_t *resident, const int32_t *pix, int64_t npix, double amb, double *out_rgba,
                   double *lo, double *hi, int32_t *out_n, int nthreads)
{
    if (V->nlevels < 1 || V->nlevels > ORC_MAX_LEVELS || V->brick < 1) return -1;
    if (mode != ORC_MOP && mode != ORC_MIP) return -1;
    if (P->level_step) return -1;
    if (!pix) npix = (int64_t)c->w * c->h;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < npix; ++i) {
        int32_t px = pix ? pix[2 * i] : (int32_t)(i % c->w);
        int32_t py = pix ? pix[2 * i + 1] : (int32_t)(i / c->w);
        orc_ray r;
        orc_make_ray(c, V->dims[0], px, py, &r);
        double kept[4] = {0.0, 0.0, 0.0, 0.0};
        double best = mode == ORC_MOP ? 0.0 : -1.0; /* MOP: largest alpha; MIP: largest x */
        int64_t n = 0;
        orc_tflookup L;
        if (r.hit) {
            for (int got; (got = sample_lookup(V, c, tf, P, resident, &r, n, &L)); ++n) {
                if (got == 2) continue;
                if (mode == ORC_MOP && L.rgba[3] > best) {
                    best = L.rgba[3];
                    memcpy(kept, L.rgba, sizeof kept);
                } else if (mode == ORC_MIP && L.x > best) {
                    best = L.x;
                }
            }
        }
        if (mode == ORC_MIP && best >= 0.0) {
            tf_at(tf, best, &L);
            memcpy(kept, L.rgba, sizeof kept);
        }
        double *o = &out_rgba[4 * i];
        composite_one(kept, P, o);
        out_n[i] = (int32_t)n;
        if (lo) {
            memcpy(&lo[4 * i], o, 4 * sizeof(double));
            memcpy(&hi[4 * i], o, 4 * sizeof(double));
            if (mode == ORC_MOP) {
                for (int64_t k = 0; k < n; ++k) {
                    if (sample_lookup(V, c, tf, P, resident, &r, k, &L) != 1) continue;
                    if (!(L.rgba[3] >= best - amb)) continue;
                    double cand[4];
                    composite_one(L.rgba, P, cand);
                    for (int ch = 0; ch < 4; ++ch) {
                        if (cand[ch] < lo[4 * i + ch]) lo[4 * i + ch] = cand[ch];
                        if (cand[ch] > hi[4 * i + ch]) hi[4 * i + ch] = cand[ch];
                    }
                }
            }
        }
    }
    return 0;
}

/* --------------------------------------------------------- adjoint */

/*
 * Adjoint of one level of the box filter (orc_downsample), for gradients with respect to
 * the finer level: each coarse voxel c hands g_coarse[c] / 8 to each of its 8 children
 * 2c + d, d in {0,1}^3, a child index beyond the fine edge replaced by the last fine voxel
 * exactly as the filter replaces it (so an edge voxel can receive several shares).  The
 * filter is the mean of the children; for integer storage its rounding is taken as the mean
 * (its derivative is 1/8 per child almost everywhere).  Accumulates into g_fine.
 */
void orc_downsample_transpose(const int64_t Dfine[3], const double *g_coarse, double *g_fine)
{
    int64_t Dc[3];
    for (int a = 0; a < 3; ++a) Dc[a] = (Dfine[a] + 1) / 2;
    for (int64_t z = 0; z < Dc[2]; ++z)
        for (int64_t y = 0; y < Dc[1]; ++y)
            for (int64_t x = 0; x < Dc[0]; ++x) {
                const double share = g_coarse[x + Dc[0] * (y + Dc[1] * z)] / 8.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            int64_t cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                            if (cx > Dfine[0] - 1) cx = Dfine[0] - 1;
                            if (cy > Dfine[1] - 1) cy = Dfine[1] - 1;
                            if (cz > Dfine[2] - 1) cz = Dfine[2] - 1;
                            g_fine[cx + Dfine[0] * (cy + Dfine[1] * cz)] += share;
                        }
            }
}

/*
 * Gradient of L with respect to the transfer function and to the normalised
 * voxel values of level 0, given dL/dI per pixel (I = output RGBA).  Not in
 * the paper (which does not differentiate); it is the exact derivative of the
 * compositing sum above, samples in reverse order:
 *   R <- bg;  for k = n-1 .. 0:
 *     dL/dalpha_k = T_k * sum_ch g_ch (c_k,ch - R_ch)     (alpha: c = 1)
 *     dL/dc_k,ch  = g_ch * T_k * alpha_k
 *     R_ch <- alpha_k c_k,ch + (1 - alpha_k) R_ch
 * then through the TF lerp (weights 1 - w, w; dv = 255 * (tf[i+1] - tf[i]) .
 * d, zero when the clamp is active) and the trilinear weights to the voxels.
 * The early-termination index n is held fixed (alt_select[i] = 1 flips the
 * ambiguous decision as in orc_render).  T_k here are plain float64 products.
 * With footprint LOD a sample on level l contributes to the voxels of level l,
 * and each level's gradient reaches level 0 through the adjoint of the box filter
 * that made the level (orc_downsample_transpose), coarsest level first.
 * dtf [256][4] and dvox [level-0 voxels] are float64 and are accumulated into (+=).
 */
int orc_render_grad(const orc_volume *V, const orc_camera *c, const float *tf, const orc_params *P,
                    const int32_t *pix, int64_t npix, double amb, const double *dI,
                    const int32_t *alt_select, double *dtf, double *dvox, int nthreads)
{
    if (P->level_step) return -1;
    if (!pix) npix = (int64_t)c->w * c->h;
    /* per-level gradients, levels laid end to end */
    int64_t lvoff[ORC_MAX_LEVELS + 1];
    lvoff[0] = 0;
    for (int l = 0; l < V->nlevels; ++l) lvoff[l + 1] = lvoff[l] + V->dims[l][0] * V->dims[l][1] * V->dims[l][2];
    const int64_t nvox = lvoff[V->nlevels];
    const float scale = lod_scale(c);
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#endif
    double *pdtf = calloc((size_t)nt * 1024, sizeof(double));
    double **pvox = calloc((size_t)nt, sizeof(double *));
    if (!pdtf || !pvox) return -2;
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mydtf = pdtf + 1024 * tid;
        double *myvox = calloc((size_t)nvox, sizeof(double));
        pvox[tid] = myvox;
        int64_t cap = 0;
        orc_interp *Is = NULL;
        orc_tflookup *Ls = NULL;
        double *Ts = NULL;
        int *Lv = NULL;
        if (!myvox) err = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < npix; ++i) {
            if (!myvox) continue;
            int32_t px = pix ? pix[2 * i] : (int32_t)(i % c->w);
            int32_t py = pix ? pix[2 * i + 1] : (int32_t)(i / c->w);
            orc_ray r;
            orc_make_ray(c, V->dims[0], px, py, &r);
            orc_state S;
            int64_t ak;
            int64_t n = march(V, c, tf, P, NULL, &r, -1, amb, &ak, &S);
            if (alt_select && alt_select[i] && ak >= 0) n = march(V, c, tf, P, NULL, &r, ak, amb, NULL, &S);
            if (n == 0) continue;
            if (n > cap) {
                cap = n;
                Is = realloc(Is, sizeof(orc_interp) * cap);
                Ls = realloc(Ls, sizeof(orc_tflookup) * cap);
                Ts = realloc(Ts, sizeof(double) * cap);
                Lv = realloc(Lv, sizeof(int) * cap);
            }
            /* forward again, keeping every sample */
            double T = 1.0;
            for (int64_t k = 0; k < n; ++k) {
                float t = sample_t(&r, P->step, k);
                float p[3];
                for (int a = 0; a < 3; ++a) p[a] = r.o[a] + t * r.d[a];
                Lv[k] = lod_level(t, scale, P->lod_bias, V->nlevels, P->lod_mode);
                orc_resolve R;
                resolve(V, Lv[k], p, &R);
                interp(V, &R, &Is[k]);
                tf_lookup(tf, Is[k].v, &Ls[k]);
                Ts[k] = T;
                T *= (1.0 - Ls[k].rgba[3]);
            }
            const double *g = &dI[4 * i];
            double Rr[4] = {P->bg[0], P->bg[1], P->bg[2], P->bg[3]};
            for (int64_t k = n - 1; k >= 0; --k) {
                const orc_tflookup *L = &Ls[k];
                double al = L->rgba[3];
                double c4[4] = {L->rgba[0], L->rgba[1], L->rgba[2], 1.0};
                double dal = 0.0;
                for (int ch = 0; ch < 4; ++ch) dal += g[ch] * (c4[ch] - Rr[ch]);
                dal *= Ts[k];
                double drgba[4];
                for (int ch = 0; ch < 3; ++ch) drgba[ch] = g[ch] * Ts[k] * al;
                drgba[3] = dal;
                double dv = 0.0;
                for (int ch = 0; ch < 4; ++ch) {
                    mydtf[4 * L->i + ch] += (1.0 - L->w) * drgba[ch];
                    mydtf[4 * (L->i + 1) + ch] += L->w * drgba[ch];
                    dv += drgba[ch] * ((double)tf[4 * (L->i + 1) + ch] - (double)tf[4 * L->i + ch]);
                }
                dv = L->inside ? 255.0 * dv : 0.0;
                for (int q = 0; q < 8; ++q) myvox[lvoff[Lv[k]] + Is[k].corner[q]] += Is[k].cw[q] * dv;
                for (int ch = 0; ch < 4; ++ch) Rr[ch] = al * c4[ch] + (1.0 - al) * Rr[ch];
            }
        }
        free(Is);
        free(Ls);
        free(Ts);
        free(Lv);
    }
    double *gsum = calloc((size_t)nvox, sizeof(double));
    if (!gsum) err = 1;
    for (int t = 0; t < nt; ++t) {
        for (int j = 0; j < 1024; ++j) dtf[j] += pdtf[1024 * t + j];
        if (pvox[t]) {
            if (gsum)
                for (int64_t j = 0; j < nvox; ++j) gsum[j] += pvox[t][j];
            free(pvox[t]);
        }
    }
    if (gsum) {
        /* coarsest level first: each level's gradient onto the level it was filtered from */
        for (int l = V->nlevels - 1; l >= 1; --l)
            orc_downsample_transpose(V->dims[l - 1], gsum + lvoff[l], gsum + lvoff[l - 1]);
        for (int64_t j = 0; j < lvoff[1]; ++j) dvox[j] += gsum[j];
        free(gsum);
    }
    free(pvox);
    free(pdtf);
    return err ? -2 : 0;
}

/* ray setup exported for tests */
int orc_ray_info(const orc_camera *c, const int64_t D0[3], int32_t px, int32_t py, float *out /* o3 d3 t0 t1 */,
                 int32_t *hit)
{
    orc_ray r;
    orc_make_ray(c, D0, px, py, &r);
    for (int a = 0; a < 3; ++a) {
        out[a] = r.o[a];
        out[3 + a] = r.d[a];
    }
    out[6] = r.t0;
    out[7] = r.t1;
    *hit = r.hit;
    return 0;
}

/* LOD level of a sample at depth t (exported for tests). */
int orc_lod_level(const orc_camera *c, float t, int bias, int nlevels, int mode)
{
    return lod_level(t, lod_scale(c), bias, nlevels, mode);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
