/*
 * synth.c -- seeded synthetic inputs for the bricked raycaster.
 *
 * This module only MAKES INPUTS: voxel volumes drawn from a counter-based
 * generator (splitmix64, Steele/Lea/Flood 2014).  It holds none of the
 * rendering arithmetic (no rays, no resolve, no interpolation rule used by the
 * method, no transfer function, no compositing).  Both the CUDA path and the
 * CPU oracle consume what it writes; neither imports the other.
 *
 * The paper benchmarks on two datasets that are not available here (a 4352^3
 * float32 Mandelbulb and a 1634x12723x9070 uint16 light-sheet scan, Sec. IV-A,
 * Table I) and on procedurally generated on-demand volumes (Sec. V-C).  The
 * generators below stand in for them with the same kind of structure: smooth
 * blobs plus noise, and fractal value noise with embedded spheres.
 *
 * Layout of every dense output: x fastest, then y, then z
 * (index = x + Dx*(y + Dy*z)).  Voxel i has its centre at i + 0.5.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- counter-based random numbers ------------------------------------- */

static inline uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* A keyed draw: stream selects the purpose, ctr the item. */
static inline uint64_t draw64(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return splitmix64(splitmix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + ctr);
}

static inline double draw01(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return (double)(draw64(seed, stream, ctr) >> 11) * 0x1.0p-53;
}

enum {
    ST_BLOB = 1,
    ST_NOISE = 2,
    ST_LATTICE = 3,
    ST_SPHERE = 4,
};

/* Exported for the determinism tests. */
double synth_draw01(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return draw01(seed, stream, ctr);
}

/* ---- Gaussian blobs + uniform noise ----------------------------------- */

/*
 * value(x) = min(vmax, sum_b amp_b * exp(-|x - c_b|^2 / (2 sigma_b^2)) + noise(x))
 * noise(x) ~ U[0, noise_hi) drawn per voxel from (seed, linear index).
 * Blob b: centre U[0,D) per axis, sigma U[sig_lo, sig_hi], amp U[amp_lo, amp_hi].
 * dtype 0: stored as uint8 floor(value) (vmax should be 255);
 * dtype 3: stored as float32 (value rounded once).
 * The Gaussian is separable, so each blob keeps one 1D table per axis.
 */
int synth_blobs(int dtype, const int64_t D[3], uint64_t seed, int nblobs,
                double sig_lo, double sig_hi, double amp_lo, double amp_hi,
                double noise_hi, double vmax, void *out, int nthreads)
{
    if (dtype != 0 && dtype != 3) return -1;
    if (nblobs < 0 || nblobs > 4096) return -1;
    const int64_t Dx = D[0], Dy = D[1], Dz = D[2];
    if (Dx <= 0 || Dy <= 0 || Dz <= 0) return -1;
    double *amp = malloc(sizeof(double) * (nblobs ? nblobs : 1));
    double **tab = malloc(sizeof(double *) * 3 * (nblobs ? nblobs : 1));
    if (!amp || !tab) return -2;
    for (int b = 0; b < nblobs; ++b) {
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = draw01(seed, ST_BLOB, 8 * b + a) * (double)D[a];
        double sig = sig_lo + (sig_hi - sig_lo) * draw01(seed, ST_BLOB, 8 * b + 3);
        amp[b] = amp_lo + (amp_hi - amp_lo) * draw01(seed, ST_BLOB, 8 * b + 4);
        for (int a = 0; a < 3; ++a) {
            double *t = malloc(sizeof(double) * D[a]);
            if (!t) return -2;
            for (int64_t i = 0; i < D[a]; ++i) {
                double dx = ((double)i + 0.5) - c[a];
                t[i] = exp(-(dx * dx) / (2.0 * sig * sig));
            }
            tab[3 * b + a] = t;
        }
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t z = 0; z < Dz; ++z) {
        for (int64_t y = 0; y < Dy; ++y) {
            double *fy = malloc(sizeof(double) * (nblobs ? nblobs : 1));
            for (int b = 0; b < nblobs; ++b) fy[b] = amp[b] * tab[3 * b + 1][y] * tab[3 * b + 2][z];
            const int64_t row = Dx * (y + Dy * z);
            for (int64_t x = 0; x < Dx; ++x) {
                double s = 0.0;
                for (int b = 0; b < nblobs; ++b) s += fy[b] * tab[3 * b][x];
                s += noise_hi * draw01(seed, ST_NOISE, (uint64_t)(row + x));
                if (s > vmax) s = vmax;
                if (dtype == 0) {
                    ((uint8_t *)out)[row + x] = (uint8_t)floor(s);
                } else {
                    ((float *)out)[row + x] = (float)s;
                }
            }
            free(fy);
        }
    }
    for (int b = 0; b < 3 * nblobs; ++b) free(tab[b]);
    free(tab);
    free(amp);
    return 0;
}

/* ---- fractal value noise + spheres ------------------------------------ */

static inline double smooth01(double f) { return f * f * (3.0 - 2.0 * f); }

/* The value at lattice point (ix, iy, iz) of octave oct is draw01(seed, ST_LATTICE + 16 oct,
 * key(ix, iy, iz)).  draw01 hashes the (seed, stream) pair first; that hash is taken once per
 * octave (lattice_stream) and the point's draw finished from it (lattice_h). */
static inline uint64_t lattice_stream(uint64_t seed, int oct)
{
    return splitmix64(seed ^ ((ST_LATTICE + 16 * (uint64_t)oct) * 0xD1B54A32D192ED03ull));
}

static inline double lattice_h(uint64_t h_oct, int64_t ix, int64_t iy, int64_t iz)
{
    uint64_t key = ((uint64_t)(ix & 0x1FFFFF)) | ((uint64_t)(iy & 0x1FFFFF) << 21) |
                   ((uint64_t)(iz & 0x1FFFFF) << 42);
    return (double)(splitmix64(h_oct + key) >> 11) * 0x1.0p-53;
}

typedef struct {
    double c[3], r, v;
} sphere_t;

/*
 * Region generator for the noise + spheres volume.
 *
 * The level-0 field f(p), p in level-0 voxel units, is
 *   f(p) = sum_o g^o * vn_o(p / P_o) / sum_o g^o,  P_o = period0 / 2^o, g = 0.5,
 * with vn_o a value noise (hashed lattice values, smoothstep-weighted
 * trilinear blend), overridden inside spheres (|p - c| <= r -> sphere value;
 * later spheres win).
 *
 * A region at level `level` holds voxels i = origin + idx for idx in
 * [0, extent) per axis, clamped to [0, Dl-1] (edge replicate), each sampled at
 * its centre p = (i + 0.5) * spacing.  At coarse levels octaves whose period is
 * below 2*spacing are replaced by their mean 0.5, so each level is a smoothed
 * version of the field (this is how procedural on-demand bricks define levels).
 * Output: uint16 round(f * 65535), x fastest.
 */
static int region_impl(const int64_t D0[3], int level, const int64_t Dl[3], const int64_t origin[3],
                       const int64_t extent[3], uint64_t seed, int octaves, double period0, int nspheres,
                       double r_lo, double r_hi, double v_lo, double v_hi, void *out, int out8, int nthreads);

int synth_noise_spheres_region(const int64_t D0[3], int level, const int64_t Dl[3],
                               const int64_t origin[3], const int64_t extent[3],
                               uint64_t seed, int octaves, double period0, int nspheres,
                               double r_lo, double r_hi, double v_lo, double v_hi,
                               uint16_t *out, int nthreads)
{
    return region_impl(D0, level, Dl, origin, extent, seed, octaves, period0, nspheres, r_lo, r_hi, v_lo, v_hi,
                       out, 0, nthreads);
}

/* The same field stored as uint8 round(f * 255). */
int synth_noise_spheres_region8(const int64_t D0[3], int level, const int64_t Dl[3],
                                const int64_t origin[3], const int64_t extent[3],
                                uint64_t seed, int octaves, double period0, int nspheres,
                                double r_lo, double r_hi, double v_lo, double v_hi,
                                uint8_t *out, int nthreads)
{
    return region_impl(D0, level, Dl, origin, extent, seed, octaves, period0, nspheres, r_lo, r_hi, v_lo, v_hi,
                       out, 1, nthreads);
}

/*
 * Brick source for on-demand loading: the parameters of a noise + spheres volume and its
 * brick grid.  synth_brick_provider() fills n bricks of (B+1)^3 voxels each (the brick plus
 * one voxel on its +x/+y/+z sides, indices clamped to the level), bricks in parallel.
 * reqs[n][4] = level, bx, by, bz.  Level l has ceil(D_{l-1} / 2) voxels per axis and every
 * level is generated directly from the field (see region_impl).  Returns 0 on success.
 */
typedef struct {
    int64_t D0[3];
    int32_t brick, levels, out8, nthreads;
    uint64_t seed;
    int32_t octaves, nspheres;
    double period0, r_lo, r_hi, v_lo, v_hi;
} synth_brick_source;

int synth_brick_provider(void *user, int n, const int32_t *reqs, void *dst)
{
    const synth_brick_source *S = (const synth_brick_source *)user;
    const int64_t B1 = S->brick + 1;
    const int64_t nvox = B1 * B1 * B1;
    int err = 0;
#ifdef _OPENMP
    if (S->nthreads > 0) omp_set_num_threads(S->nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int i = 0; i < n; ++i) {
        const int level = reqs[4 * i];
        if (level < 0 || level >= S->levels) {
            err |= 1;
            continue;
        }
        int64_t Dl[3], origin[3], extent[3] = {B1, B1, B1};
        for (int a = 0; a < 3; ++a) {
            Dl[a] = S->D0[a];
            for (int l = 0; l < level; ++l) Dl[a] = (Dl[a] + 1) / 2;
            origin[a] = (int64_t)reqs[4 * i + 1 + a] * S->brick;
        }
        void *o = (char *)dst + (size_t)i * (size_t)nvox * (S->out8 ? 1 : 2);
        err |= region_impl(S->D0, level, Dl, origin, extent, S->seed, S->octaves, S->period0, S->nspheres, S->r_lo,
                           S->r_hi, S->v_lo, S->v_hi, o, S->out8, 1) != 0;
    }
    return err;
}

static int region_impl(const int64_t D0[3], int level, const int64_t Dl[3], const int64_t origin[3],
                       const int64_t extent[3], uint64_t seed, int octaves, double period0, int nspheres,
                       double r_lo, double r_hi, double v_lo, double v_hi, void *out, int out8, int nthreads)
{
    if (octaves < 1 || octaves > 16 || nspheres < 0 || level < 0) return -1;
    double sp[3];
    for (int a = 0; a < 3; ++a) {
        if (D0[a] <= 0 || Dl[a] <= 0 || extent[a] <= 0) return -1;
        sp[a] = (double)D0[a] / (double)Dl[a];
    }
    sphere_t *sph = malloc(sizeof(sphere_t) * (nspheres ? nspheres : 1));
    if (!sph) return -2;
    for (int s = 0; s < nspheres; ++s) {
        for (int a = 0; a < 3; ++a) sph[s].c[a] = draw01(seed, ST_SPHERE, 8 * s + a) * (double)D0[a];
        sph[s].r = r_lo + (r_hi - r_lo) * draw01(seed, ST_SPHERE, 8 * s + 3);
        sph[s].v = v_lo + (v_hi - v_lo) * draw01(seed, ST_SPHERE, 8 * s + 4);
    }
    double gsum = 0.0, g = 1.0;
    for (int o = 0; o < octaves; ++o) { gsum += g; g *= 0.5; }
    const double smin = fmin(sp[0], fmin(sp[1], sp[2]));
    const int64_t Ex = extent[0], Ey = extent[1], Ez = extent[2];
    /* positions per axis (clamped index -> centre in level-0 units) */
    double *pos[3];
    for (int a = 0; a < 3; ++a) {
        pos[a] = malloc(sizeof(double) * extent[a]);
        for (int64_t i = 0; i < extent[a]; ++i) {
            int64_t gi = origin[a] + i;
            if (gi < 0) gi = 0;
            if (gi > Dl[a] - 1) gi = Dl[a] - 1;
            pos[a][i] = ((double)gi + 0.5) * sp[a];
        }
    }
    /* the spheres that can reach the region: the box of its voxel centres against each sphere's
     * bounding box, widened far beyond rounding so that no sphere the exact tests below could
     * accept is dropped (kept in their order: later spheres win) */
    int *near = malloc(sizeof(int) * (nspheres ? nspheres : 1));
    int nnear = 0;
    for (int s = 0; s < nspheres; ++s) {
        int in = 1;
        for (int a = 0; a < 3 && in; ++a) {
            const double rw = sph[s].r * (1.0 + 1e-9) + 1e-9;
            in = sph[s].c[a] + rw >= pos[a][0] && sph[s].c[a] - rw <= pos[a][extent[a] - 1];
        }
        if (in) near[nnear++] = s;
    }
    /* per octave and x: the lattice cell and the blend weight along x (they do not depend on y
     * or z, so every row of the region reuses them) */
    int64_t *cellx = malloc(sizeof(int64_t) * (size_t)octaves * (size_t)Ex);
    double *wxt = malloc(sizeof(double) * (size_t)octaves * (size_t)Ex);
    int64_t ncolmax = 2;
    for (int o = 0; o < octaves; ++o) {
        const double P = period0 / (double)(1 << o);
        for (int64_t x = 0; x < Ex; ++x) {
            const double fx0 = pos[0][x] / P;
            const int64_t ix = (int64_t)floor(fx0);
            cellx[(size_t)o * Ex + x] = ix;
            wxt[(size_t)o * Ex + x] = smooth01(fx0 - (double)ix);
        }
        const int64_t nc = cellx[(size_t)o * Ex + Ex - 1] - cellx[(size_t)o * Ex] + 2;
        if (nc > ncolmax) ncolmax = nc;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t z = 0; z < Ez; ++z) {
        double *acc = malloc(sizeof(double) * Ex);
        /* per octave: the lattice values at the region's columns ix0 .. ix1 + 1 for the current
         * cell row (iy, iz) -- l00, l10, l01, l11 -- refilled when iy changes, and their blend
         * along y and z for the current row */
        double *lat = malloc(sizeof(double) * 4 * (size_t)octaves * (size_t)ncolmax);
        double *ecol = malloc(sizeof(double) * (size_t)ncolmax);
        int64_t lat_iy[16];
        for (int o = 0; o < octaves; ++o) lat_iy[o] = INT64_MIN;
        int *cand = malloc(sizeof(int) * (nspheres ? nspheres : 1));
        const double pz = pos[2][z];
        int ncand = 0;
        for (int q = 0; q < nnear; ++q) {
            const int s = near[q];
            if (fabs(pz - sph[s].c[2]) <= sph[s].r) cand[ncand++] = s;
        }
        for (int64_t y = 0; y < Ey; ++y) {
            const double py = pos[1][y];
            for (int64_t x = 0; x < Ex; ++x) acc[x] = 0.0;
            double gw = 1.0;
            for (int o = 0; o < octaves; ++o, gw *= 0.5) {
                const double P = period0 / (double)(1 << o);
                if (P < 2.0 * smin) {
                    for (int64_t x = 0; x < Ex; ++x) acc[x] += gw * 0.5;
                    continue;
                }
                const double fy0 = py / P, fz0 = pz / P;
                const int64_t iy = (int64_t)floor(fy0), iz = (int64_t)floor(fz0);
                const double wy = smooth01(fy0 - (double)iy), wz = smooth01(fz0 - (double)iz);
                const int64_t *cx = cellx + (size_t)o * Ex;
                const double *wxo = wxt + (size_t)o * Ex;
                const int64_t ix0 = cx[0], ncol = cx[Ex - 1] - ix0 + 2;  /* cellx rises with x */
                double *L = lat + 4 * (size_t)o * (size_t)ncolmax;
                if (iy != lat_iy[o]) {
                    const uint64_t h_oct = lattice_stream(seed, o);
                    for (int64_t c = 0; c < ncol; ++c) {
                        L[4 * c + 0] = lattice_h(h_oct, ix0 + c, iy, iz);
                        L[4 * c + 1] = lattice_h(h_oct, ix0 + c, iy + 1, iz);
                        L[4 * c + 2] = lattice_h(h_oct, ix0 + c, iy, iz + 1);
                        L[4 * c + 3] = lattice_h(h_oct, ix0 + c, iy + 1, iz + 1);
                    }
                    lat_iy[o] = iy;
                }
                for (int64_t c = 0; c < ncol; ++c) {
                    const double l00 = L[4 * c + 0], l10 = L[4 * c + 1], l01 = L[4 * c + 2], l11 = L[4 * c + 3];
                    const double a0 = l00 + wy * (l10 - l00);
                    const double a1 = l01 + wy * (l11 - l01);
                    ecol[c] = a0 + wz * (a1 - a0);
                }
                for (int64_t x = 0; x < Ex; ++x) {
                    const int64_t c = cx[x] - ix0;
                    const double e0 = ecol[c], e1 = ecol[c + 1];
                    acc[x] += gw * (e0 + wxo[x] * (e1 - e0));
                }
            }
            for (int64_t x = 0; x < Ex; ++x) acc[x] /= gsum;
            for (int c = 0; c < ncand; ++c) {
                const sphere_t *s = &sph[cand[c]];
                const double dy = py - s->c[1], dz = pz - s->c[2];
                const double rr = s->r * s->r - dy * dy - dz * dz;
                if (rr < 0) continue;
                /* candidate x range from the chord, widened by 2; the exact test decides */
                const double half = sqrt(rr);
                int64_t xlo = (int64_t)floor((s->c[0] - half) / sp[0] - 0.5) - origin[0] - 2;
                int64_t xhi = (int64_t)ceil((s->c[0] + half) / sp[0] - 0.5) - origin[0] + 2;
                if (xlo < 0) xlo = 0;
                if (xhi > Ex - 1) xhi = Ex - 1;
                if (origin[0] < 0 || origin[0] + Ex > Dl[0]) { xlo = 0; xhi = Ex - 1; }
                for (int64_t x = xlo; x <= xhi; ++x) {
                    const double dx = pos[0][x] - s->c[0];
                    if (dx * dx + dy * dy + dz * dz <= s->r * s->r) acc[x] = s->v;
                }
            }
            const int64_t ro = Ex * (y + Ey * z);
            for (int64_t x = 0; x < Ex; ++x) {
                double v = acc[x];
                if (v < 0) v = 0;
                if (v > 1) v = 1;
                if (out8)
                    ((uint8_t *)out)[ro + x] = (uint8_t)floor(v * 255.0 + 0.5);
                else
                    ((uint16_t *)out)[ro + x] = (uint16_t)floor(v * 65535.0 + 0.5);
            }
        }
        free(cand);
        free(ecol);
        free(lat);
        free(acc);
    }
    for (int a = 0; a < 3; ++a) free(pos[a]);
    free(cellx);
    free(wxt);
    free(near);
    free(sph);
    return 0;
}
