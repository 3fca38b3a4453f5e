// render_common.cuh -- device building blocks of the raycaster and the persistent forward
// kernel template k_render, shared by the translation units that instantiate its variants
// (kernels_render.cu: emission/absorption, with and without gradient checkpoints;
// kernels_project.cu: maximum-opacity and maximum-intensity projection).
//
// The forward kernel is the data-parallel hot path of the bricked multi-resolution
// raycaster (Drees & Risse, "Palace", Sec. III-E, III-H, IV-A, V-C): per pixel it builds
// the camera ray, intersects the volume box, and for each sample picks the LOD level from
// the pixel footprint, resolves the brick through the level's page table into the atlas,
// interpolates trilinearly inside the brick (the +side apron makes every corner local),
// maps the value through the RGBA transfer function, and composites front to back with
// early termination.
//
// Work distribution: one persistent grid; each warp takes ray tiles (or, on a resume
// pass, chunks of 32 suspended rays) from a global counter and refills lanes whose ray
// ended as soon as fewer than `refill_thresh` lanes are busy, so early-terminated rays do
// not leave lanes idle.
//
// Decision arithmetic (ray setup, sample positions, LOD level, voxel index, brick id) is
// binary32 with explicit round-to-nearest intrinsics, so it never contracts into FMAs and
// is bit-identical to any correct IEEE binary32 evaluation of the same expressions.
#pragma once
#include "internal.cuh"

namespace volrc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__host__ __device__ constexpr int log2i(int x) { return x <= 1 ? 0 : 1 + log2i(x / 2); }

template <int DT>
struct Voxel;
template <>
struct Voxel<VOL_U8> {
    using T = uint8_t;
    static __device__ __forceinline__ float ld(const T* p) { return (float)__ldg(p); }
};
template <>
struct Voxel<VOL_U16> {
    using T = uint16_t;
    static __device__ __forceinline__ float ld(const T* p) { return (float)__ldg(p); }
};
template <>
struct Voxel<VOL_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
};
template <>
struct Voxel<VOL_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T* p) { return __ldg(p); }
};

// Transfer-function coordinate x = 255 * clamp(v_normalised, 0, 1) from an interpolated
// stored value (u8: stored = 255 v; u16: stored = 65535 v; floats: v).
template <int DT>
__device__ __forceinline__ float tf_coord(float v) {
    if (DT == VOL_U8) return v;
    if (DT == VOL_U16) return v * (255.0f / 65535.0f);
    return fminf(fmaxf(v, 0.0f), 1.0f) * 255.0f;
}
template <int DT>
__device__ __forceinline__ bool tf_inside(float v) {
    if (DT == VOL_U8 || DT == VOL_U16) return true;
    return v >= 0.0f && v <= 1.0f;
}

struct Ray {
    float o[3], d[3], t0, t1;
    bool hit;
};

// Pixel -> ray and slab entry/exit against [0, D0) (Fig. 1 entry_exit_points).
__device__ __forceinline__ void make_ray(const ViewDev& V, const float D0f[3], int px, int py, Ray& r) {
    const float u = __fsub_rn(__fmul_rn(__fdiv_rn(__fadd_rn((float)px, 0.5f), (float)V.w), 2.0f), 1.0f);
    const float v = __fsub_rn(1.0f, __fmul_rn(__fdiv_rn(__fadd_rn((float)py, 0.5f), (float)V.h), 2.0f));
    const float cx = __fmul_rn(u, V.tan_aspect);
    const float cy = __fmul_rn(v, V.tan);
    float dd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        dd[a] = __fadd_rn(__fadd_rn(V.fwd[a], __fmul_rn(cx, V.right[a])), __fmul_rn(cy, V.up[a]));
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(dd[0], dd[0]), __fmul_rn(dd[1], dd[1])), __fmul_rn(dd[2], dd[2]));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(len2));
    float t0 = 0.0f, t1 = __int_as_float(0x7f800000);
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.d[a] = __fmul_rn(dd[a], inv);
        r.o[a] = V.eye[a];
        if (r.d[a] == 0.0f) {
            if (r.o[a] < 0.0f || r.o[a] >= D0f[a]) hit = false;
            continue;
        }
        const float ta = __fdiv_rn(__fsub_rn(0.0f, r.o[a]), r.d[a]);
        const float tb = __fdiv_rn(__fsub_rn(D0f[a], r.o[a]), r.d[a]);
        const float tn = ta < tb ? ta : tb;
        const float tf = ta < tb ? tb : ta;
        if (tn > t0) t0 = tn;
        if (tf < t1) t1 = tf;
    }
    r.t0 = t0;
    r.t1 = t1;
    r.hit = hit && (t0 < t1);
}

// Footprint LOD (Sec. V-C): l = clamp(ilogb(t * lodscale) + bias, 0, L-1); l = 0 when the
// footprint has no normal exponent.  t >= 0 and lodscale > 0, so q has a clear sign bit and its
// exponent field is the exponent + 127; +0 and subnormals have field 0, giving -127 as required.
__device__ __forceinline__ int lod_level(float t, float lodscale, int bias, int nlevels) {
    const float q = __fmul_rn(t, lodscale);
    const int e = (int)(__float_as_uint(q) >> 23) - 127;
    return min(max(e + bias, 0), nlevels - 1);
}

struct Resolved {
    int i0[3];
    float w[3];
    uint32_t pti;   // page-table index (level offset + brick id)
    uint32_t local; // element offset inside the slot
};

// One level's constants, held in registers by the render loop.
struct LvReg {
    float r[3];     // D_l / D_0 per axis (binary32)
    float Dm[3];    // D_l - 1 per axis, as floats (exact: D_l <= 2^24)
    int nb0, nb1;   // bricks along x and y
    uint32_t off;   // first page-table entry of the level (sparse table: of its top grid)
    int tn0, tn1;   // sparse table: top-grid entries along x and y
};

__device__ __forceinline__ LvReg load_lv(const LevelDev& L) {
    LvReg R;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.r[a] = L.r[a];
        R.Dm[a] = (float)(L.D[a] - 1);
    }
    R.nb0 = L.nb[0];
    R.nb1 = L.nb[1];
    R.off = L.pt_off;
    R.tn0 = L.tn[0];
    R.tn1 = L.tn[1];
    return R;
}

// Sparse page table: the top-grid entry of brick (h0, h1, h2) on a level, and its position
// inside the middle and leaf pages (packed: 8 low bits per axis).
__device__ __forceinline__ uint32_t sparse_top(const LvReg& L, int h0, int h1, int h2) {
    constexpr int s = 2 * kPageShift;
    return L.off + (uint32_t)(((h2 >> s) * L.tn1 + (h1 >> s)) * L.tn0 + (h0 >> s));
}
__device__ __forceinline__ uint32_t sparse_sub(int h0, int h1, int h2) {
    return ((uint32_t)(h2 & 255) << 16) | ((uint32_t)(h1 & 255) << 8) | (uint32_t)(h0 & 255);
}
__device__ __forceinline__ uint32_t sparse_mid_local(uint32_t sub) {
    constexpr int p = kPageShift, m = (1 << kPageShift) - 1;
    return (((sub >> (16 + p)) & m) << (2 * p)) | (((sub >> (8 + p)) & m) << p) | ((sub >> p) & m);
}
__device__ __forceinline__ uint32_t sparse_leaf_local(uint32_t sub) {
    constexpr int p = kPageShift, m = (1 << kPageShift) - 1;
    return (((sub >> 16) & m) << (2 * p)) | (((sub >> 8) & m) << p) | (sub & m);
}
// Slot of the brick through the three levels (kInvalidSlot when a page or the brick is
// absent); leaf receives the leaf entry's pool index (the brick's identity) or kInvalidSlot.
__device__ __forceinline__ uint32_t sparse_walk(const uint32_t* __restrict__ pool, const LvReg& L, int h0, int h1, int h2,
                                                uint32_t& leaf) {
    leaf = kInvalidSlot;
    const uint32_t sub = sparse_sub(h0, h1, h2);
    const uint32_t m = __ldg(pool + sparse_top(L, h0, h1, h2));
    if (m == kInvalidSlot) return kInvalidSlot;
    const uint32_t f = __ldg(pool + m + sparse_mid_local(sub));
    if (f == kInvalidSlot) return kInvalidSlot;
    leaf = f + sparse_leaf_local(sub);
    return __ldg(pool + leaf);
}

// Grid position on a level, clamp to edge, chunk addressing (Sec. III-A).
// local = element (compact: row = B+1) or entry (quad: row = B) offset inside the slot.
// Clamp to edge: i = floor(x) < 0 gives i0 = 0 and weight 0, i >= D_l - 1 gives i0 = D_l - 1 and
// weight 0, else i0 = i and weight x - i.  Clamping x itself to [0, D_l - 1] first gives exactly
// these (x below 0 becomes 0, x at or past D_l - 1 becomes D_l - 1, both with zero fraction)
// without a branch.
__device__ __forceinline__ void resolve_reg(const LvReg& L, int bshift, int bmask, int row, const float p[3],
                                            Resolved& R) {
    int h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = __fsub_rn(__fmul_rn(p[a], L.r[a]), 0.5f);
        const float xc = fminf(fmaxf(x, 0.0f), L.Dm[a]);
        const float fx = floorf(xc);
        R.i0[a] = (int)fx;
        R.w[a] = __fsub_rn(xc, fx);
        h[a] = R.i0[a] >> bshift;
        l[a] = R.i0[a] & bmask;
    }
    R.pti = L.off + (uint32_t)(h[0] + L.nb0 * (h[1] + L.nb1 * h[2]));
    R.local = (uint32_t)((l[2] * row + l[1]) * row + l[0]);
}

__device__ __forceinline__ void resolve(const LevelDev& L, int bshift, int bmask, int row, const float p[3],
                                        Resolved& R) {
    resolve_reg(load_lv(L), bshift, bmask, row, p, R);
}

// Trilinear interpolation of the 8 corners at atlas element `base` (+x, +y, +z neighbours
// at +1, +B1, +B1^2 thanks to the apron).
template <int DT, int BS = 0>
__device__ __forceinline__ float trilinear(const typename Voxel<DT>::T* a, unsigned long long base, int B1_rt,
                                           const float w[3]) {
    const int B1 = BS ? BS + 1 : B1_rt;
    const unsigned long long sy = (unsigned long long)B1, sz = (unsigned long long)B1 * B1;
    const float v000 = Voxel<DT>::ld(a + base), v100 = Voxel<DT>::ld(a + base + 1);
    const float v010 = Voxel<DT>::ld(a + base + sy), v110 = Voxel<DT>::ld(a + base + sy + 1);
    const float v001 = Voxel<DT>::ld(a + base + sz), v101 = Voxel<DT>::ld(a + base + sz + 1);
    const float v011 = Voxel<DT>::ld(a + base + sz + sy), v111 = Voxel<DT>::ld(a + base + sz + sy + 1);
    const float c00 = fmaf(w[0], v100 - v000, v000);
    const float c10 = fmaf(w[0], v110 - v010, v010);
    const float c01 = fmaf(w[0], v101 - v001, v001);
    const float c11 = fmaf(w[0], v111 - v011, v011);
    const float c0 = fmaf(w[1], c10 - c00, c00);
    const float c1 = fmaf(w[1], c11 - c01, c01);
    return fmaf(w[2], c1 - c0, c0);
}

// Quad layout: entry e holds the voxels (x, y), (x+1, y), (x, y+1), (x+1, y+1) of one slice;
// the entry of slice z+1 is B*B entries further.  Same interpolation order as trilinear().
template <int DT>
struct QuadEntry;
template <>
struct QuadEntry<VOL_U8> {
    using V = unsigned int;
    static __device__ __forceinline__ void get(V q, float v[4]) {
        v[0] = (float)(q & 0xFFu);
        v[1] = (float)((q >> 8) & 0xFFu);
        v[2] = (float)((q >> 16) & 0xFFu);
        v[3] = (float)(q >> 24);
    }
};
template <>
struct QuadEntry<VOL_U16> {
    using V = uint2;
    static __device__ __forceinline__ void get(V q, float v[4]) {
        v[0] = (float)(q.x & 0xFFFFu);
        v[1] = (float)(q.x >> 16);
        v[2] = (float)(q.y & 0xFFFFu);
        v[3] = (float)(q.y >> 16);
    }
};
template <>
struct QuadEntry<VOL_F16> {
    using V = uint2;
    static __device__ __forceinline__ void get(V q, float v[4]) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
};
template <>
struct QuadEntry<VOL_F32> {
    using V = float4;
    static __device__ __forceinline__ void get(V q, float v[4]) {
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    }
};

template <int DT, int BS = 0>
__device__ __forceinline__ float trilinear_quad(const void* atlas, unsigned long long entry, int B_rt, const float w[3]) {
    using Q = QuadEntry<DT>;
    const int B = BS ? BS : B_rt;
    const typename Q::V* a = (const typename Q::V*)atlas;
    float e0[4], e1[4];
    Q::get(__ldg(a + entry), e0);
    Q::get(__ldg(a + entry + (unsigned long long)(B * B)), e1);
    const float c00 = fmaf(w[0], e0[1] - e0[0], e0[0]);
    const float c10 = fmaf(w[0], e0[3] - e0[2], e0[2]);
    const float c01 = fmaf(w[0], e1[1] - e1[0], e1[0]);
    const float c11 = fmaf(w[0], e1[3] - e1[2], e1[2]);
    const float c0 = fmaf(w[1], c10 - c00, c00);
    const float c1 = fmaf(w[1], c11 - c01, c01);
    return fmaf(w[2], c1 - c0, c0);
}

// Either layout: `base` is the slot's element offset plus local (compact) or its entry offset
// plus local (quad).
template <int DT, int BS, bool Q>
__device__ __forceinline__ float sample_value(const void* atlas, unsigned long long base, int B1, const float w[3]) {
    if constexpr (Q) return trilinear_quad<DT, BS>(atlas, base, B1 - 1, w);
    else return trilinear<DT, BS>((const typename Voxel<DT>::T*)atlas, base, B1, w);
}

// TF entries i0..i1 that lookups at coordinates in [x0, x1] touch, with one entry of margin
// on each side for the last-bit rounding of the interpolation, clamped to 0..255.  False when
// the range is empty or not a number (the brick is then never skipped).
__device__ __forceinline__ bool entry_span(float x0, float x1, int& i0, int& i1) {
    if (!(x0 <= x1)) return false;
    i0 = (int)fminf(fmaxf(x0 - 1.0f, 0.0f), 255.0f);
    i1 = (int)fminf(fmaxf(x1 + 2.0f, 0.0f), 255.0f);
    return true;
}

// A brick whose stored values lie in [rng.x, rng.y] has zero opacity at every sample when no
// TF entry that a lookup in that range can touch (the same margin as entry_span) has non-zero
// alpha.  tf_coord maps every stored value (floats clamped, +-inf included) into [0, 255], so
// the indices stay within 0..256 even for the unordered range (+inf, -inf) of an all-NaN slot.
template <int DT>
__device__ __forceinline__ bool brick_empty(float2 rng, const int* s_apre) {
    const float xlo = tf_coord<DT>(rng.x), xhi = tf_coord<DT>(rng.y);
    const int ilo = max((int)xlo - 1, 0), ihi = min((int)xhi + 2, 255);
    return s_apre[ihi + 1] - s_apre[ilo] == 0;
}

// Range of TF coordinates that trilinear samples of a brick with stored values in
// [rng.x, rng.y] can take.  Integer values interpolate without rounding past the corner
// values; for floating-point ones each of the three lerp levels may overshoot by an ulp, so
// the range is widened by 4 ulps of the largest magnitude.
template <int DT>
__device__ __forceinline__ float2 coord_range(float2 rng) {
    if (DT == VOL_F16 || DT == VOL_F32) {
        const float m = fmaxf(fabsf(rng.x), fabsf(rng.y)) * 5e-7f;
        rng.x -= m;
        rng.y += m;
    }
    return make_float2(tf_coord<DT>(rng.x), tf_coord<DT>(rng.y));
}

// Largest TF opacity over entries lo..hi (0 <= lo <= hi <= 255) from the sparse table s_amx:
// levels j = 0..8, entry i of level j the maximum over entries i .. min(i + 2^j - 1, 255).
__device__ __forceinline__ float tf_alpha_max(const float* s_amx, int lo, int hi) {
    const int j = 31 - __clz(hi - lo + 1);
    return fmaxf(s_amx[j * 256 + lo], s_amx[j * 256 + hi - (1 << j) + 1]);
}

// MOP: no sample of the brick can have opacity above `kept`, so none can replace the kept
// sample (a later one replaces it only when strictly more opaque).  The bound is raised by
// 2^-22 relative for the rounding of the interpolation between entries.
template <int DT>
__device__ __forceinline__ bool brick_below_alpha(float2 rng, const float* s_amx, float kept) {
    const float2 x = coord_range<DT>(rng);
    int ilo, ihi;
    if (!entry_span(x.x, x.y, ilo, ihi)) return false;
    const float b = tf_alpha_max(s_amx, ilo, ihi);
    return fmaf(fabsf(b), 2.4e-7f, b) <= kept;
}

// MIP: no sample of the brick can have a TF coordinate above the kept maximum.
template <int DT>
__device__ __forceinline__ bool brick_below_coord(float2 rng, float kept) {
    return coord_range<DT>(rng).y <= kept;
}

// Macro-cell index of a clamped voxel inside its brick (cells of 2^cs voxels, 2^cb per axis).
__device__ __forceinline__ uint32_t cell_of(const int i0[3], int bmask, int cs, int cb) {
    return ((uint32_t)((i0[2] & bmask) >> cs) << (2 * cb)) | ((uint32_t)((i0[1] & bmask) >> cs) << cb) |
           (uint32_t)((i0[0] & bmask) >> cs);
}

// Quad layout with a brick edge BS >= 8 known at compile time: a sample's local entry offset is
// (z BS + y) BS + x, so its macro-cell (2^cb per axis, cells of BS >> cb voxels) is a fixed set
// of bits of it: key() keeps those bits (equal keys: the same cell of the brick), index() packs
// them into the cell's table index (cz CB + cy) CB + cx, CB = 2^cb.
template <int BS>
struct CellBits {
    static constexpr int bs = BS >= 8 ? log2i(BS) : 3;  // (only used for BS >= 8)
    static constexpr int cb = cell_bits_for(bs), cs = bs - cb;
    static constexpr uint32_t cm = (1u << cb) - 1u;
    static constexpr uint32_t field = ((1u << bs) - 1u) & ~((1u << cs) - 1u);
    static constexpr uint32_t mask = field | (field << bs) | (field << (2 * bs));
    static __device__ __forceinline__ uint32_t key(uint32_t loc) { return loc & mask; }
    static __device__ __forceinline__ uint32_t index(uint32_t key) {
        return ((key >> cs) & cm) | ((key >> (bs + cs - cb)) & (cm << cb)) | ((key >> (2 * bs + cs - 2 * cb)) & (cm << (2 * cb)));
    }
};

// A macro-cell whose TF-entry span is [span & 255, span >> 8] holds no sample that changes the
// lane's state (the per-cell form of brick_empty / brick_below_alpha / brick_below_coord; the
// span already carries the one-entry margins).  MIP: every coordinate in the cell is below the
// span's upper entry.
template <int MODE>
__device__ __forceinline__ bool span_skippable(uint32_t span, const int* s_apre, const float* s_amx, float kept) {
    const int lo = (int)(span & 255u), hi = (int)(span >> 8);
    if (MODE == kMop) {
        const float b = tf_alpha_max(s_amx, lo, hi);
        return fmaf(fabsf(b), 2.4e-7f, b) <= kept;
    }
    if (MODE == kMip) return (float)hi <= kept;
    return s_apre[hi + 1] - s_apre[lo] == 0;
}

// The brick form of the same test, from the slot's value range.
template <int DT, int MODE>
__device__ __forceinline__ bool brick_skippable(float2 rng, const int* s_apre, const float* s_amx, float kept) {
    if (MODE == kMop) return brick_below_alpha<DT>(rng, s_amx, kept);
    if (MODE == kMip) return brick_below_coord<DT>(rng, kept);
    return brick_empty<DT>(rng, s_apre);
}

// Decision record of sample k for the block searches below: its level and clamped voxel.
struct SampleKey {
    bool valid;  // t_k < t1
    int l;
    Resolved R;
};

template <bool LOD>
__device__ __forceinline__ SampleKey sample_key(int k, const float o[3], const float d[3], float t0, float t1, float step,
                                                float lodscale, int bias, int nlev, const LevelDev* s_lv, int bshift,
                                                int bmask, int row) {
    SampleKey K;
    const float t = __fadd_rn(t0, __fmul_rn((float)k, step));
    K.valid = t < t1;
    const float p[3] = {__fadd_rn(o[0], __fmul_rn(t, d[0])), __fadd_rn(o[1], __fmul_rn(t, d[1])),
                        __fadd_rn(o[2], __fmul_rn(t, d[2]))};
    K.l = LOD ? lod_level(t, lodscale, bias, nlev) : 0;
    resolve(s_lv[K.l], bshift, bmask, row, p, K.R);
    return K;
}

// Estimated last sample of the ray in the block of sample k (key K): the block is the level and
// the voxel index >> shift on every axis (shift = log2 B: the brick; log2 M: the macro-cell).
// Samples of one block are contiguous along a ray (level and clamped voxel indices are monotone
// in t), and the block ends at its exit face or at the next LOD switch, whichever comes first.
// Reciprocals are approximate: the caller verifies the estimate with the exact decision
// arithmetic (the batch that starts at the estimate checks that its first sample is in the block).
template <bool LOD>
__device__ __forceinline__ int block_end_estimate(int k, const SampleKey& K, int shift, const float o[3],
                                                  const float d[3], float t0, float t1, float step, float lodscale,
                                                  int bias, int nlev, const LevelDev* s_lv) {
    const LevelDev& L = s_lv[K.l];
    float te = t1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int g = K.R.i0[a] >> shift;
        if (d[a] > 0.0f && ((g + 1) << shift) <= L.D[a] - 1)
            te = fminf(te, __fdividef(((float)((g + 1) << shift) + 0.5f) * L.ir[a] - o[a], d[a]));
        else if (d[a] < 0.0f && g > 0)
            te = fminf(te, __fdividef(((float)(g << shift) + 0.5f) * L.ir[a] - o[a], d[a]));
    }
    if (LOD && K.l < nlev - 1) {  // the level rises once t * lodscale reaches 2^(l + 1 - bias)
        const int e = K.l + 1 - bias;
        if (e <= -126) te = 0.0f;  // (only at t = 0: no jump)
        else if (e < 127) te = fminf(te, __fdividef(__int_as_float((e + 127) << 23), lodscale));
    }
    const float est = __fdividef(te - t0, step);
    return est > (float)k && est < 16777216.0f ? (int)est : k;
}

// Last sample of the ray that resolves to the same page-table entry (level and brick) as
// sample k_start: estimated from the brick's exit faces (and the next LOD switch), then fixed
// by the exact decision arithmetic.  Samples with one page-table entry are contiguous along a
// ray (level, voxel and brick indices are monotone in t).
template <bool LOD>
__device__ __noinline__ int brick_last_sample(int k_start, uint32_t pti_start, const float o[3], const float d[3],
                                              float t0, float t1, float step, float lodscale, int bias, int nlev,
                                              const LevelDev* s_lv, int bshift, int bmask, int row, int B) {
    auto pti_of = [&](int k) -> uint32_t {
        const float t = __fadd_rn(t0, __fmul_rn((float)k, step));
        if (!(t < t1)) return kInvalidSlot;
        const float p[3] = {__fadd_rn(o[0], __fmul_rn(t, d[0])), __fadd_rn(o[1], __fmul_rn(t, d[1])),
                            __fadd_rn(o[2], __fmul_rn(t, d[2]))};
        const int l = LOD ? lod_level(t, lodscale, bias, nlev) : 0;
        Resolved R;
        resolve(s_lv[l], bshift, bmask, row, p, R);
        return R.pti;
    };
    const float ts = __fadd_rn(t0, __fmul_rn((float)k_start, step));
    const float ps[3] = {__fadd_rn(o[0], __fmul_rn(ts, d[0])), __fadd_rn(o[1], __fmul_rn(ts, d[1])),
                         __fadd_rn(o[2], __fmul_rn(ts, d[2]))};
    const int l = LOD ? lod_level(ts, lodscale, bias, nlev) : 0;
    const LevelDev& L = s_lv[l];
    Resolved R;
    resolve(L, bshift, bmask, row, ps, R);
    float te = t1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int h = R.i0[a] >> bshift;
        if (d[a] > 0.0f && h < L.nb[a] - 1) te = fminf(te, (((float)((h + 1) * B) + 0.5f) / L.r[a] - o[a]) / d[a]);
        else if (d[a] < 0.0f && h > 0) te = fminf(te, (((float)(h * B) + 0.5f) / L.r[a] - o[a]) / d[a]);
    }
    if (LOD && l < nlev - 1) te = fminf(te, ldexpf(1.0f, l + 1 - bias) / lodscale);
    int ke = max(k_start, (int)floorf((te - t0) / step));
    for (int s = 0; s < 8 && ke > k_start && pti_of(ke) != pti_start; ++s) --ke;
    if (pti_of(ke) != pti_start) ke = k_start;
    for (int s = 0; s < 8 && pti_of(ke + 1) == pti_start; ++s) ++ke;
    return ke;
}

// Progressive preview (Sec. III-H: a low-resolution image from coarser levels first): the
// sample at depth t, whose brick on its level is not resident, on the finest coarser level
// whose brick at the same position is resident.  ok = false when no level is.
struct Fallback {
    uint32_t slot, local;
    float w[3];
    bool ok;
};

template <bool LOD, bool SP>
__device__ __noinline__ Fallback preview_fallback(const uint32_t* __restrict__ pt, float t, float o0, float o1,
                                                  float o2, float d0, float d1, float d2, float lodscale, int bias,
                                                  int nlev, const LevelDev* s_lv, int bshift, int bmask, int row) {
    Fallback F;
    F.ok = false;
    F.slot = 0;
    F.local = 0;
    F.w[0] = F.w[1] = F.w[2] = 0.0f;
    const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)),
                        __fadd_rn(o2, __fmul_rn(t, d2))};
    const int l = LOD ? lod_level(t, lodscale, bias, nlev) : 0;
    for (int m = l + 1; m < nlev; ++m) {
        Resolved R;
        resolve(s_lv[m], bshift, bmask, row, p, R);
        uint32_t leaf;
        const uint32_t s = SP ? sparse_walk(pt, load_lv(s_lv[m]), R.i0[0] >> bshift, R.i0[1] >> bshift,
                                            R.i0[2] >> bshift, leaf)
                              : __ldg(pt + R.pti);
        if (s != kInvalidSlot) {
            F.ok = true;
            F.slot = s;
            F.local = R.local;
            F.w[0] = R.w[0];
            F.w[1] = R.w[1];
            F.w[2] = R.w[2];
            break;
        }
    }
    return F;
}

__device__ __forceinline__ int find_view_tile(const ViewDev* views, int nviews, int item) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_off <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_ray(const ViewDev* views, int nviews, long long ray) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].ray_off <= ray) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t hash_key(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Records a brick request (Sec. III-H): insert key into the open-addressing table with
// bounded linear probing; a newly inserted key is appended to the request list with one
// atomic per group of inserting lanes.
__device__ __forceinline__ void request_brick(const RenderDev& P, uint32_t key) {
    uint32_t h = hash_key(key) & P.req_cap_mask;
    int state = 2;  // 0 new, 1 present, 2 overflow
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const uint32_t prev = atomicCAS(&P.req_table[h], 0u, key);
        if (prev == 0u) { state = 0; break; }
        if (prev == key) { state = 1; break; }
        h = (h + 1) & P.req_cap_mask;
    }
    if (state == 2) atomicAdd(&P.counters[kReqOverflow], 1u);
    const unsigned m = __activemask();
    const unsigned mnew = __ballot_sync(m, state == 0);
    if (state == 0) {
        const int leader = __ffs(mnew) - 1;
        const unsigned lane = threadIdx.x & 31;
        unsigned base = 0;
        if ((int)lane == leader) base = atomicAdd(&P.counters[kReqCount], (unsigned)__popc(mnew));
        base = __shfl_sync(mnew, base, leader);
        const unsigned pos = base + __popc(mnew & ((1u << lane) - 1));
        if (pos < P.req_list_cap) P.req_list[pos] = key;
        else atomicAdd(&P.counters[kReqOverflow], 1u);
    }
}

// request_brick for the sparse page table: the key is (level << 60 | bz << 40 | by << 20 | bx) + 1.
__device__ __forceinline__ void request_brick64(const RenderDev& P, unsigned long long key) {
    uint32_t h = hash_key((uint32_t)key ^ hash_key((uint32_t)(key >> 32))) & P.req_cap_mask;
    int state = 2;  // 0 new, 1 present, 2 overflow
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const unsigned long long prev = atomicCAS(&P.req_table64[h], 0ull, key);
        if (prev == 0ull) { state = 0; break; }
        if (prev == key) { state = 1; break; }
        h = (h + 1) & P.req_cap_mask;
    }
    if (state == 2) atomicAdd(&P.counters[kReqOverflow], 1u);
    const unsigned m = __activemask();
    const unsigned mnew = __ballot_sync(m, state == 0);
    if (state == 0) {
        const int leader = __ffs(mnew) - 1;
        const unsigned lane = threadIdx.x & 31;
        unsigned base = 0;
        if ((int)lane == leader) base = atomicAdd(&P.counters[kReqCount], (unsigned)__popc(mnew));
        base = __shfl_sync(mnew, base, leader);
        const unsigned pos = base + __popc(mnew & ((1u << lane) - 1));
        if (pos < P.req_list_cap) P.req_list64[pos] = key;
        else atomicAdd(&P.counters[kReqOverflow], 1u);
    }
}

// Look-ahead for a ray about to wait for brick miss_pti (sample k): request the next P.prefetch
// bricks along the ray as well (those not resident), so that the resumed ray does not wait a
// round for each of them.
template <bool LOD>
__device__ __noinline__ void prefetch_next_brick(const RenderDev& P, int k, uint32_t miss_pti, float o0, float o1,
                                                 float o2, float d0, float d1, float d2, float t0, float t1,
                                                 float lodscale, const LevelDev* s_lv, int bshift, int bmask, int row,
                                                 int B) {
    const float o3[3] = {o0, o1, o2}, d3[3] = {d0, d1, d2};
    const int nlev = P.vol.nlevels;
    uint32_t cur = miss_pti;
    int kc = k;
    for (int ahead = 0; ahead < P.prefetch; ++ahead) {
        const int kl = brick_last_sample<LOD>(kc, cur, o3, d3, t0, t1, P.step, lodscale, P.lod_bias, nlev, s_lv, bshift,
                                              bmask, row, B);
        kc = kl + 1;
        const float tn = __fadd_rn(t0, __fmul_rn((float)kc, P.step));
        if (!(tn < t1)) return;
        const float pn[3] = {__fadd_rn(o0, __fmul_rn(tn, d0)), __fadd_rn(o1, __fmul_rn(tn, d1)),
                             __fadd_rn(o2, __fmul_rn(tn, d2))};
        const int ln = LOD ? lod_level(tn, lodscale, P.lod_bias, nlev) : 0;
        Resolved R;
        resolve(s_lv[ln], bshift, bmask, row, pn, R);
        if (R.pti == cur) return;  // no progress (cannot happen past the brick's last sample)
        cur = R.pti;
        if (__ldg(P.vol.pt + cur) == kInvalidSlot) request_brick(P, cur + 1u);
    }
}

// Sparse page table: the request key of the sample at depth t (its level and brick).
template <bool LOD>
__device__ __noinline__ unsigned long long sparse_request_key(float t, float o0, float o1, float o2, float d0, float d1,
                                                             float d2, float lodscale, int bias, int nlev,
                                                             const LevelDev* s_lv, int bshift, int bmask, int row) {
    const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)), __fadd_rn(o2, __fmul_rn(t, d2))};
    const int l = LOD ? lod_level(t, lodscale, bias, nlev) : 0;
    Resolved R;
    resolve(s_lv[l], bshift, bmask, row, p, R);
    return (((unsigned long long)l << 60) | ((unsigned long long)(R.i0[2] >> bshift) << 40) |
            ((unsigned long long)(R.i0[1] >> bshift) << 20) | (unsigned long long)(R.i0[0] >> bshift)) + 1ull;
}

__device__ __forceinline__ void suspend_ray(const RenderDev& P, long long ray, int k, float C0, float C1, float C2,
                                            float T, float tk) {
    const unsigned m = __activemask();
    const int leader = __ffs(m) - 1;
    const unsigned lane = threadIdx.x & 31;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(&P.counters[kSuspCount], (unsigned)__popc(m));
    base = __shfl_sync(m, base, leader);
    const unsigned pos = base + __popc(m & ((1u << lane) - 1));
    if ((long long)pos < P.nrays) {
        SuspRec r;
        r.ray = ray;
        r.k = k;
        r.tk_bits = __float_as_int(tk);
        r.C[0] = C0;
        r.C[1] = C1;
        r.C[2] = C2;
        r.T = T;
        P.susp_out[pos] = r;
    } else {
        atomicAdd(&P.counters[kDevError], 1u);
    }
}

// Value tape (gradient mode): sample k of a ray at [(k / 32) * nrays + ray] * 32 + k % 32.
__device__ __forceinline__ long long tape_at(long long nrays, long long ray, int k) {
    return ((long long)(k >> kCkptShift) * nrays + ray) * kCkptEvery + (k & (kCkptEvery - 1));
}

// Writes the values of samples kfrom .. k-1 still held in the lane's staging group tb (tb.w the
// value of sample k-1, tb.z of k-2, tb.y of k-3; samples before kfrom are not the lane's).
__device__ __forceinline__ void tape_flush(float* tape, long long nrays, long long ray, int k, int kfrom, float4 tb) {
    const int q = k & 3;
    if (q >= 1 && k - 1 >= kfrom) tape[tape_at(nrays, ray, k - 1)] = tb.w;
    if (q >= 2 && k - 2 >= kfrom) tape[tape_at(nrays, ray, k - 2)] = tb.z;
    if (q >= 3 && k - 3 >= kfrom) tape[tape_at(nrays, ray, k - 3)] = tb.y;
}

// Samples per lane per loop iteration: their page-table lookups and gathers are issued together,
// then composited in order (memory-level parallelism along one ray).
#ifndef VOLRC_BATCH
#define VOLRC_BATCH 6
#endif
// Level-scaled sampling carries the depths and levels of its batch: 5 samples measured faster.
#ifndef VOLRC_BATCH_LS
#define VOLRC_BATCH_LS 5
#endif
// Empty-space skipping keeps the tested block's value range and span through the batch.
#ifndef VOLRC_BATCH_ES
#define VOLRC_BATCH_ES 6
#endif
constexpr int kBatchDefault = VOLRC_BATCH;
constexpr int kBatchLevelStep = VOLRC_BATCH_LS;
constexpr int kBatchSkip = VOLRC_BATCH_ES;
// Minimum resident CTAs per SM the register allocation must allow.
#ifndef VOLRC_MIN_CTAS
#define VOLRC_MIN_CTAS 5
#endif


// The TF row of one sample: weight wt, entry a = tf[i] and dab = tf[i+1] - tf[i] at the TF
// coordinate of the interpolated value (i = min(floor(x), 254)).
template <int DT>
__device__ __forceinline__ void tf_index(float val, int& i, float& wt) {
    const float x = tf_coord<DT>(val);
    i = min((int)x, 254);
    wt = x - (float)i;
}

template <int DT>
__device__ __forceinline__ void tf_row(float val, const float4* s_tf, const float4* s_tfd, float& wt, float4& a,
                                       float4& dab) {
    int i;
    tf_index<DT>(val, i, wt);
    a = s_tf[i];
    dab = s_tfd[i];
}

// One sample's compositing step for mode MODE (not MIP) from its TF row (lane state C0..C2, T as
// k_render keeps it); returns true when the ray may stop after it.  Split from the row read so
// that a batch's rows can be read before any of its samples is composited.
template <int MODE, bool LS = false>
__device__ __forceinline__ bool composite_row(float wt, float4 a, float4 dab, float amax_tf, float et, float& T,
                                              float& C0, float& C1, float& C2, int l = 0) {
    static_assert(MODE != kMip, "MIP composites the TF coordinate");
    const float al = fmaf(wt, dab.w, a.w);
    if (MODE == kMop) {
        if (al > T) {  // the first sample of largest opacity is kept
            T = al;
            C0 = fmaf(wt, dab.x, a.x);
            C1 = fmaf(wt, dab.y, a.y);
            C2 = fmaf(wt, dab.z, a.z);
        }
        return T >= amax_tf;
    }
    if (LS && l > 0) {
        // level-scaled step: the sample stands for 2^l reference steps, 1 - a' = (1 - a)^(2^l)
        float om = 1.0f - al;
        for (int q = 0; q < l; ++q) om = om * om;
        const float Ta = T * (1.0f - om);
        C0 = fmaf(Ta, fmaf(wt, dab.x, a.x), C0);
        C1 = fmaf(Ta, fmaf(wt, dab.y, a.y), C1);
        C2 = fmaf(Ta, fmaf(wt, dab.z, a.z), C2);
        T = T * om;
        return __fsub_rn(1.0f, T) >= et;
    }
    const float Ta = T * al;
    C0 = fmaf(Ta, fmaf(wt, dab.x, a.x), C0);
    C1 = fmaf(Ta, fmaf(wt, dab.y, a.y), C1);
    C2 = fmaf(Ta, fmaf(wt, dab.z, a.z), C2);
    T = T * (1.0f - al);
    return __fsub_rn(1.0f, T) >= et;
}

// One sample's compositing step from its interpolated value, any mode.
template <int DT, int MODE, bool LS = false>
__device__ __forceinline__ bool composite_sample(float val, const float4* s_tf, const float4* s_tfd, float amax_tf,
                                                 float et, float& T, float& C0, float& C1, float& C2, int l = 0) {
    if constexpr (MODE == kMip) {
        const float x = tf_coord<DT>(val);
        if (x > T) T = x;
        return T >= 255.0f;  // no coordinate lies above 255
    } else {
        float wt;
        float4 a, dab;
        tf_row<DT>(val, s_tf, s_tfd, wt, a, dab);
        return composite_row<MODE, LS>(wt, a, dab, amax_tf, et, T, C0, C1, C2, l);
    }
}

// Depth of sample k: the kept depth under level-scaled sampling, else t0 + k dt.
__device__ __forceinline__ float tcur_or_t(bool ls, float tcur, float t0, int k, float step) {
    return ls ? tcur : __fadd_rn(t0, __fmul_rn((float)k, step));
}

// Level-scaled sampling: the sample after one at t on level l lies dt * 2^l further (the
// scaling by an exact power of two does not round).
__device__ __forceinline__ float next_t_level_step(float t, float step, int l) {
    return __fadd_rn(t, __fmul_rn(step, (float)(1 << l)));
}

// Tail of the persistent launch: once the work queue is empty and at most kAssistLanes rays are
// left in a warp, the warp's lanes split among those rays -- G lanes per ray, G = 2, 4 or 8 --
// and lane q of a group decides, looks up and interpolates samples k + 6 q .. k + 6 q + 5 of its
// group's ray; the group's first lane composites all 6 G of them in order, taking each one's TF
// index and weight from its lane by shuffle.  The decisions, values and compositing are the
// per-sample arithmetic of the main loop, in the same order, so the image and the sample counts
// are bit for bit the same; the longest rays of a frame (often ~30 times the mean) then end in
// about 1/G of the iterations instead of running on alone while their SM idles.  Any compositing
// mode but the gradient one, on a resident volume (no requests, preview, level-scaled steps,
// sparse table or skipping); called by all 32 lanes of the warp.
#ifndef VOLRC_ASSIST_LANES
#define VOLRC_ASSIST_LANES 16
#endif
constexpr int kAssistLanes = VOLRC_ASSIST_LANES;
constexpr int kAssistBatch = 6;
// Tiles wholly outside a view's bound of the volume's projection are written as misses without
// setting up their rays.
#ifndef VOLRC_CULL_TILES
#define VOLRC_CULL_TILES 1
#endif
constexpr bool kCullTiles = VOLRC_CULL_TILES != 0;

// The misses of a ray tile that cannot meet the volume, written by the lanes of a warp (not
// inlined: it keeps the render loop's code as it is).
__device__ __noinline__ void write_missed_tile(const RenderDev& P, const ViewDev& V, int x0, int y0, int cnt, int lane) {
    for (int q = lane; q < cnt; q += 32) {
        const int px = x0 + q % P.tile_w, py = y0 + q / P.tile_w;
        if (px < V.w && py < V.h) {
            const long long r = V.ray_off + (long long)py * V.w + px;
            P.out[r] = P.bg;
            if (P.nsamp) P.nsamp[r] = 0;
            if (P.ray_n) P.ray_n[r] = 0;
        }
    }
}

template <int DT, bool LOD, int MODE, int BS, bool Q>
__device__ __noinline__ void assist_finish(const RenderDev& P, bool live, long long ray, int tile, float o0, float o1,
                                           float o2, float d0, float d1, float d2, float t0, float t1, float lodscale,
                                           int k, float C0, float C1, float C2, float T, const float4* s_tf,
                                           const float4* s_tfd, const LevelDev* s_lv, float amax_tf) {
    constexpr int kB = kAssistBatch;
    const int lane = (int)(threadIdx.x & 31);
    const int bshift = BS ? log2i(BS) : P.vol.bshift;
    const int bmask = BS ? BS - 1 : P.vol.bmask;
    const int B1 = BS ? BS + 1 : P.vol.B1;
    const int row = Q ? B1 - 1 : B1;
    const unsigned long long slot_stride = Q ? P.vol.slot_entries : P.vol.slot_elems;
    const float step = P.step, et = P.et;
    const int nlev = P.vol.nlevels;
    int cur_l = 0;
    LvReg L = load_lv(s_lv[0]);
    for (;;) {
        // ---- groups: the r-th ray (r-th lane with one) goes to lanes r G .. r G + G - 1
        const unsigned own = __ballot_sync(kFull, live);
        if (!own) return;
        const int nr = __popc(own);
        const int G = nr <= 4 ? 8 : (nr <= 8 ? 4 : 2);
        const int r = lane / G, q = lane - r * G, gl = r * G;
        unsigned m = own;
        for (int i = 0; i < r && m; ++i) m &= m - 1u;
        const int src = m ? __ffs(m) - 1 : 0;
        const bool in = r < nr;
        o0 = __shfl_sync(kFull, o0, src); o1 = __shfl_sync(kFull, o1, src); o2 = __shfl_sync(kFull, o2, src);
        d0 = __shfl_sync(kFull, d0, src); d1 = __shfl_sync(kFull, d1, src); d2 = __shfl_sync(kFull, d2, src);
        t0 = __shfl_sync(kFull, t0, src); t1 = __shfl_sync(kFull, t1, src);
        lodscale = __shfl_sync(kFull, lodscale, src);
        k = __shfl_sync(kFull, k, src);
        C0 = __shfl_sync(kFull, C0, src); C1 = __shfl_sync(kFull, C1, src); C2 = __shfl_sync(kFull, C2, src);
        T = __shfl_sync(kFull, T, src);
        ray = __shfl_sync(kFull, ray, src);
        tile = __shfl_sync(kFull, tile, src);
        live = in;
        // ---- march until a group's ray ends (then the rays are regrouped)
        bool ended = false;
        while (!__any_sync(kFull, ended)) {
            uint32_t pti[kB], loc[kB], slot[kB];
            float wgt[kB][3];
            int nvalid = live ? kB : 0;
            const float kf = (float)(k + kB * q);  // exact: indices stay below 2^24
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const float t = __fadd_rn(t0, __fmul_rn(__fadd_rn(kf, (float)j), step));
                if (!(t < t1) && nvalid == kB) nvalid = j;
                const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)),
                                    __fadd_rn(o2, __fmul_rn(t, d2))};
                if (LOD) {
                    const int l = lod_level(t, lodscale, P.lod_bias, nlev);
                    if (l != cur_l) {
                        cur_l = l;
                        L = load_lv(s_lv[l]);
                    }
                }
                Resolved R;
                resolve_reg(L, bshift, bmask, row, p, R);
                pti[j] = R.pti;
                loc[j] = R.local;
                wgt[j][0] = R.w[0];
                wgt[j][1] = R.w[1];
                wgt[j][2] = R.w[2];
            }
#pragma unroll
            for (int j = 0; j < kB; ++j) slot[j] = __ldg(P.vol.pt + (j < nvalid ? pti[j] : 0u));
            int miss_at = kB;
#pragma unroll
            for (int j = kB - 1; j >= 0; --j)
                if (j < nvalid && slot[j] == kInvalidSlot) miss_at = j;
            // usage stamps (idempotent: every lane stamps the bricks of its own samples)
#pragma unroll
            for (int j = 0; j < kB; ++j)
                if (P.last_used && j < nvalid && j < miss_at && (j == 0 || pti[j] != pti[j - 1]))
                    P.last_used[slot[j]] = P.frame;
            int ti[kB];    // TF row (MIP: unused)
            float tw[kB];  // its weight (MIP: the TF coordinate)
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const bool use = j < nvalid && j < miss_at;
                const unsigned long long base = use ? (unsigned long long)slot[j] * slot_stride + loc[j] : 0ull;
                const float v = sample_value<DT, BS, Q>(P.vol.atlas, base, B1, wgt[j]);
                if (MODE == kMip) {
                    ti[j] = 0;
                    tw[j] = tf_coord<DT>(v);
                } else {
                    tf_index<DT>(v, ti[j], tw[j]);
                }
            }
            // ---- the group's first lane composites the group's 6 G samples in order
            bool fin = false, out = false, err = false;  // early termination, left the volume, missing brick
            int kk = k;
            for (int qq = 0; qq < G; ++qq) {
                const int from = gl + qq;  // (lanes of groups past the last ray shuffle among themselves)
                const int nv = __shfl_sync(kFull, nvalid, from), ms = __shfl_sync(kFull, miss_at, from);
#pragma unroll
                for (int j = 0; j < kB; ++j) {
                    const int tij = __shfl_sync(kFull, ti[j], from);
                    const float twj = __shfl_sync(kFull, tw[j], from);
                    if (q == 0 && live && !fin && !out && !err) {
                        if (j >= nv && nv <= ms) {
                            out = true;
                        } else if (j >= ms) {
                            err = true;
                        } else {
                            if constexpr (MODE == kMip) {
                                if (twj > T) T = twj;
                                fin = T >= 255.0f;  // no coordinate lies above 255
                            } else {
                                fin = composite_row<MODE, false>(twj, s_tf[tij], s_tfd[tij], amax_tf, et, T, C0, C1, C2);
                            }
                            ++kk;
                        }
                    }
                }
            }
            k = __shfl_sync(kFull, kk, gl);
            const bool stop = __shfl_sync(kFull, (fin || out || err) ? 1 : 0, gl) != 0;
            if (live && stop) {
                if (q == 0) {
                    if (err) {
                        atomicAdd(&P.counters[kDevError], 1u);
                    } else {
                        const float4 bg = P.bg;
                        if (MODE == kMop || MODE == kMip) {
                            // the kept sample composited once over the background, as in k_render
                            float al = 0.0f;
                            if (MODE == kMop) {
                                al = T;
                            } else if (T >= 0.0f) {  // the TF at the largest coordinate
                                const int i = min((int)T, 254);
                                const float wt = T - (float)i;
                                const float4 a = s_tf[i], dab = s_tfd[i];
                                al = fmaf(wt, dab.w, a.w);
                                C0 = fmaf(wt, dab.x, a.x);
                                C1 = fmaf(wt, dab.y, a.y);
                                C2 = fmaf(wt, dab.z, a.z);
                            }
                            const float tb = 1.0f - al;
                            P.out[ray] = make_float4(fmaf(al, C0, tb * bg.x), fmaf(al, C1, tb * bg.y),
                                                     fmaf(al, C2, tb * bg.z), fmaf(tb, bg.w, al));
                        } else {
                            P.out[ray] = make_float4(fmaf(T, bg.x, C0), fmaf(T, bg.y, C1), fmaf(T, bg.z, C2),
                                                     fmaf(T, bg.w, 1.0f - T));
                        }
                        if (P.nsamp) P.nsamp[ray] = k;
                        if (P.tile_cost && tile >= 0) atomicMax(&P.tile_cost[tile], k);
                    }
                }
                live = false;
                ended = true;
            }
        }
        if (q != 0) live = false;  // only a group's first lane keeps the ray for the regrouping
    }
}

// BS: brick edge known at compile time (32 or 64), or 0 for any power of two read at run time.
// MODE: kDvr, kDvrGrad, kMop or kMip.  Lane state (C0, C1, C2, T): emission/absorption keeps
// the partial colour and the transmittance; MOP the kept sample's colour and opacity (T,
// starting at 0); MIP the largest TF coordinate so far (T, starting at -1).
// LS: level-scaled sampling (emission/absorption only): sample k+1 lies dt * 2^l past sample k
// on level l, whose opacity is corrected to that longer step; t of the lane's next sample is
// kept in tcur (and in a suspended ray's record).
// SP: three-level sparse page table (emission/absorption, uniform steps, no empty-space jumps).
// ES: empty-space skipping: when the last sample of a batch lies in a brick or macro-cell that
// cannot change the lane's state (zero TF opacity over its value range; for MOP/MIP no opacity /
// coordinate above the kept one), the lane's next batch starts near that block's estimated last
// sample instead of the next one; the batch's first decision verifies the estimate exactly (same
// level and block), so a lane crosses a whole block per iteration in step with the other lanes of
// its warp.  One block is tested per batch, and its value range and span are loaded together with
// the gathers: a sample that enters an empty block earlier in the batch is composited (it adds
// nothing), which costs less than testing every sample.
template <int DT, bool LOD, int MODE, int BS, bool Q, bool LS = false, bool SP = false, bool ES = false>
__global__ void __launch_bounds__(kRenderThreads, VOLRC_MIN_CTAS) k_render(const __grid_constant__ RenderDev P) {
    static_assert(!LS || MODE == kDvr, "level-scaled sampling is for emission/absorption without gradients");
    static_assert(!SP || (MODE == kDvr && !LS), "the sparse page table variant is for emission/absorption");
    static_assert(!ES || (!LS && !SP), "empty-space skipping assumes uniform steps and the flat page table");
    // ES: the macro-cell of a quad-layout sample is read from its local offset; otherwise it is
    // computed from the voxel
    constexpr bool kFastCell = ES && Q && BS >= 8;
    constexpr int kBatch = LS ? kBatchLevelStep : (ES ? kBatchSkip : kBatchDefault);
    constexpr bool GRAD = MODE == kDvrGrad;
    // the tail's lane assist (assist_finish): plain emission/absorption on a resident volume
    constexpr bool kAssistOk = MODE != kDvrGrad && !LS && !SP && !ES && kAssistLanes > 0;
    const bool kAssist = kAssistOk && !P.preview && !P.req_table;
    constexpr float kT0 = MODE == kMop ? 0.0f : (MODE == kMip ? -1.0f : 1.0f);
    __shared__ float4 s_tf[256];
    __shared__ float4 s_tfd[255];  // tf[i+1] - tf[i], each difference rounded once
    __shared__ LevelDev s_lv[kMaxLevels];
    __shared__ int s_apre[257];  // s_apre[i]: TF entries below i with non-zero opacity
    __shared__ float s_amx[MODE == kMop ? 9 * 256 : 1];  // MOP: sparse max table of TF opacity
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tf[i] = P.tf[i];
    if (threadIdx.x < P.vol.nlevels) s_lv[threadIdx.x] = P.vol.lv[threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.x; i < 255; i += blockDim.x) {
        const float4 a = s_tf[i], b = s_tf[i + 1];
        s_tfd[i] = make_float4(__fsub_rn(b.x, a.x), __fsub_rn(b.y, a.y), __fsub_rn(b.z, a.z), __fsub_rn(b.w, a.w));
    }
    if (ES && threadIdx.x < 32) {
        // (only the skip tests read it) lane l counts entries 8 l .. 8 l + 7, then a scan over lanes
        const int l8 = 8 * (int)threadIdx.x;
        int c[8], tot = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = tot;
            tot += s_tf[l8 + u].w != 0.0f;
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if ((int)threadIdx.x >= o) incl += y;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s_apre[l8 + u] = incl - tot + c[u];
        if (threadIdx.x == 31) s_apre[256] = incl;
    }
    if (MODE == kMop) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_amx[i] = s_tf[i].w;
        for (int j = 1; j <= 8; ++j) {
            __syncthreads();
            for (int i = threadIdx.x; i < 256; i += blockDim.x)
                s_amx[j * 256 + i] = fmaxf(s_amx[(j - 1) * 256 + i], s_amx[(j - 1) * 256 + min(i + (1 << (j - 1)), 255)]);
        }
    }
    __syncthreads();
    // MOP stops once the kept opacity reaches the largest TF entry opacity
    const float amax_tf = MODE == kMop ? tf_alpha_max(s_amx, 0, 255) : 0.0f;

    const unsigned lane = threadIdx.x & 31;
    const unsigned ltmask = (1u << lane) - 1;
    const int bshift = BS ? log2i(BS) : P.vol.bshift;
    const int bmask = BS ? BS - 1 : P.vol.bmask;
    const int B1 = BS ? BS + 1 : P.vol.B1;
    const int row = Q ? B1 - 1 : B1;
    const unsigned long long slot_stride = Q ? P.vol.slot_entries : P.vol.slot_elems;
    const float step = P.step, et = P.et;

    // warp-uniform work pool
    int pool_next = 0, pool_cnt = 0, pool_a = 0, pool_x0 = 0, pool_y0 = 0, pool_tile = -1;
    bool queue_done = false;

    // lane state
    bool active = false;
    long long ray = 0;
    int my_tile = -1;
    float o0 = 0, o1 = 0, o2 = 0, d0 = 0, d1 = 0, d2 = 0, t0 = 0, t1 = 0, lodscale = 0;
    int k = 0;
    float C0 = 0, C1 = 0, C2 = 0, T = kT0;
    float tcur = 0.0f;  // LS: depth of sample k
    // GRAD with a value tape: the values of the current group of 4 aligned samples, and the first
    // sample this lane composited of the ray (since its start or resumption)
    float4 tb = make_float4(0.f, 0.f, 0.f, 0.f);
    int tb_from = 0;
    uint32_t cur_pti = kInvalidSlot;
    const unsigned long long ncells = ES ? 1ull << (3 * P.vol.cbits) : 0ull;
    // ES: sample k - 1 lies in a block (brick when sk_brick, else macro-cell) that cannot change
    // the lane's state
    bool sk = false, sk_brick = false;
    const int nlev = P.vol.nlevels;
    int cur_l = 0;
    LvReg L = load_lv(s_lv[0]);

    for (;;) {
        // ---- refill lanes whose ray ended
        while (!queue_done) {
            const unsigned need = __ballot_sync(kFull, !active);
            if (!need) break;
            if (pool_next >= pool_cnt) {
                int item = 0;
                if (lane == 0) item = (int)atomicAdd(&P.counters[kWork], 1u);
                item = __shfl_sync(kFull, item, 0);
                if (item >= P.nwork) {
                    queue_done = true;
                    break;
                }
                if (!P.resume) {
                    const int tile = P.tile_order ? P.tile_order[item] : item;
                    const int v = find_view_tile(P.views, P.nviews, tile);
                    const ViewDev& V = P.views[v];
                    const int tl = tile - V.tile_off;
                    const int tx = V.tiles_x;
                    pool_tile = tile;
                    pool_a = v;
                    pool_x0 = (tl % tx) * P.tile_w;
                    pool_y0 = (tl / tx) * P.tile_h;
                    pool_cnt = P.tile_w * P.tile_h;
                    if (kCullTiles &&
                        (pool_x0 > V.cx1 || pool_x0 + P.tile_w <= V.cx0 || pool_y0 > V.cy1 || pool_y0 + P.tile_h <= V.cy0)) {
                        // no ray of the tile can meet the volume (outside the view's bound of its
                        // projection): the warp writes the tile's misses at once
                        write_missed_tile(P, V, pool_x0, pool_y0, pool_cnt, (int)lane);
                        pool_next = pool_cnt;
                        continue;
                    }
                } else {
                    pool_tile = -1;
                    pool_a = item * 32;
                    pool_cnt = min(32, P.nsusp_in - item * 32);
                }
                pool_next = 0;
            }
            const int idx = pool_next + __popc(need & ltmask);
            pool_next = min(pool_cnt, pool_next + __popc(need));
            if (!active && idx < pool_cnt) {
                int view, px, py, k0 = 0;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f, tt = kT0, tk0 = 0.f;
                bool ok;
                if (!P.resume) {
                    view = pool_a;
                    px = pool_x0 + idx % P.tile_w;
                    py = pool_y0 + idx / P.tile_w;
                    ok = px < P.views[view].w && py < P.views[view].h;
                    ray = P.views[view].ray_off + (long long)py * P.views[view].w + px;
                } else {
                    const SuspRec r = P.susp_in[pool_a + idx];
                    ray = r.ray;
                    k0 = r.k;
                    c0 = r.C[0];
                    c1 = r.C[1];
                    c2 = r.C[2];
                    tt = r.T;
                    tk0 = __int_as_float(r.tk_bits);
                    view = find_view_ray(P.views, P.nviews, ray);
                    const long long loc = ray - P.views[view].ray_off;
                    px = (int)(loc % P.views[view].w);
                    py = (int)(loc / P.views[view].w);
                    ok = true;
                }
                my_tile = pool_tile;
                if (ok) {
                    Ray R;
                    make_ray(P.views[view], P.vol.D0f, px, py, R);
                    if (R.hit) {
                        active = true;
                        o0 = R.o[0]; o1 = R.o[1]; o2 = R.o[2];
                        d0 = R.d[0]; d1 = R.d[1]; d2 = R.d[2];
                        t0 = R.t0; t1 = R.t1;
                        lodscale = P.views[view].lodscale;
                        k = k0; C0 = c0; C1 = c1; C2 = c2; T = tt;
                        tb_from = k0;
                        if (LS) tcur = P.resume ? tk0 : R.t0;
                        cur_pti = kInvalidSlot;
                        sk = false;
                    } else {
                        P.out[ray] = P.bg;
                        if (P.nsamp) P.nsamp[ray] = 0;
                        if (GRAD) P.ray_n[ray] = 0;
                    }
                }
            }
        }
        unsigned act = __ballot_sync(kFull, active);
        if (!act) break;
        if constexpr (kAssistOk) {
            if (kAssist && queue_done && __popc(act) <= kAssistLanes) {
                // the tail: the warp's lanes split among its last rays (assist_finish)
                assist_finish<DT, LOD, MODE, BS, Q>(P, active, ray, my_tile, o0, o1, o2, d0, d1, d2, t0, t1, lodscale,
                                                    k, C0, C1, C2, T, s_tf, s_tfd, s_lv, amax_tf);
                break;
            }
        }

        // ---- march: per iteration up to kBatch samples of each active ray
        const int thresh = queue_done ? (kAssist ? kAssistLanes + 1 : 1) : P.refill_thresh;
        do {
            if (active) {
                // (a) decisions for the batch (ALU only)
                uint32_t pti[kBatch], loc[kBatch];
                float wgt[kBatch][3];
                int nvalid = kBatch;
                float tv[kBatch + 1];  // LS: depths of samples k .. k + kBatch
                int lv[kBatch];        // LS: their levels
                uint32_t sub[kBatch];  // SP: brick position inside the middle and leaf pages
                tv[0] = tcur;
                // ES: a lane whose sample k - 1 lies in a block that cannot change its state starts
                // the batch at the block's estimated last sample kb (verified below by sample kb)
                int kb = k;
                int key_l = 0, key_g[3] = {0, 0, 0}, key_shift = 0;  // ES: the block of sample k - 1
                if (ES && sk) {
                    const float o3[3] = {o0, o1, o2}, d3[3] = {d0, d1, d2};
                    const SampleKey K = sample_key<LOD>(k - 1, o3, d3, t0, t1, step, lodscale, P.lod_bias, nlev, s_lv,
                                                        bshift, bmask, row);
                    key_shift = sk_brick ? bshift : P.vol.cshift;
                    key_l = K.l;
                    key_g[0] = K.R.i0[0] >> key_shift;
                    key_g[1] = K.R.i0[1] >> key_shift;
                    key_g[2] = K.R.i0[2] >> key_shift;
                    // one sample short of the estimate: the batch then lands inside the block, and the
                    // block's samples at its start are passed over below
                    kb = max(k, block_end_estimate<LOD>(k - 1, K, key_shift, o3, d3, t0, t1, step, lodscale,
                                                        P.lod_bias, nlev, s_lv) - 1);
                }
                // ES: sample kb must lie in the block of sample k - 1; then every sample in between
                // does (a block's samples are contiguous along the ray) and composites nothing.  When
                // it does not (the estimate overshot), the decisions are taken again from k.
                uint32_t cell_last = 0u;  // ES: macro-cell (table index) of the batch's last sample
                for (;;) {
                    nvalid = kBatch;
                    bool in_block = true;  // ES: sample kb lies in the block of sample k
                    // sample indices as floats: (float)(k + j) = (float)k + j exactly, since the host
                    // keeps every index of a ray below 2^24 (kMaxSamplesPerRay)
                    const float kf = (float)kb;
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const float t = LS ? tv[j] : __fadd_rn(t0, __fmul_rn(__fadd_rn(kf, (float)j), step));
                        if (!(t < t1) && nvalid == kBatch) nvalid = j;
                        const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)),
                                            __fadd_rn(o2, __fmul_rn(t, d2))};
                        if (LOD) {
                            const int l = lod_level(t, lodscale, P.lod_bias, nlev);
                            if (l != cur_l) {
                                cur_l = l;
                                L = load_lv(s_lv[l]);
                            }
                        }
                        if (LS) {
                            lv[j] = LOD ? cur_l : 0;
                            tv[j + 1] = next_t_level_step(t, step, lv[j]);
                        }
                        Resolved R;
                        resolve_reg(L, bshift, bmask, row, p, R);
                        pti[j] = R.pti;
                        if (ES && j == 0)
                            in_block = (LOD ? cur_l : 0) == key_l && (R.i0[0] >> key_shift) == key_g[0] &&
                                       (R.i0[1] >> key_shift) == key_g[1] && (R.i0[2] >> key_shift) == key_g[2];
                        if (SP) {
                            const int h0 = R.i0[0] >> bshift, h1 = R.i0[1] >> bshift, h2 = R.i0[2] >> bshift;
                            pti[j] = sparse_top(L, h0, h1, h2);
                            sub[j] = sparse_sub(h0, h1, h2);
                        }
                        loc[j] = R.local;
                        if (ES && j == kBatch - 1)
                            cell_last = kFastCell ? CellBits<BS>::index(CellBits<BS>::key(R.local))
                                                  : cell_of(R.i0, bmask, P.vol.cshift, P.vol.cbits);
                        wgt[j][0] = R.w[0];
                        wgt[j][1] = R.w[1];
                        wgt[j][2] = R.w[2];
                    }
                    if (!(ES && sk && kb > k) || (nvalid > 0 && in_block)) break;
                    kb = k;
                }
                if (ES && sk && kb > k) {
                    if (GRAD) {
                        const int cs = P.ckpt_shift;
                        for (int kk = ((k + (1 << cs) - 1) >> cs) << cs; kk < kb; kk += 1 << cs)
                            if (kk > 0) P.ckpt[(long long)((kk >> cs) - 1) * P.nrays + ray] = T;
                    }
                    {  // count the samples jumped over (one atomic per warp)
                        const unsigned m = __activemask();
                        const unsigned long long tot = __reduce_add_sync(m, (unsigned)(kb - k));
                        if ((int)lane == __ffs(m) - 1)
                            atomicAdd(reinterpret_cast<unsigned long long*>(P.counters + kSkipped), tot);
                    }
                    k = kb;
                }
                sk = false;
                // (b) page-table lookups, all issued together (samples past the exit read entry 0)
                uint32_t slot[kBatch];
                if (SP) {
                    // three dependent lookups, each issued for the whole batch; pti becomes the leaf
                    // entry (the brick's identity) of resident bricks
                    uint32_t e[kBatch];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) e[j] = j < nvalid ? __ldg(P.vol.pt + pti[j]) : kInvalidSlot;
#pragma unroll
                    for (int j = 0; j < kBatch; ++j)
                        e[j] = e[j] != kInvalidSlot ? __ldg(P.vol.pt + e[j] + sparse_mid_local(sub[j])) : kInvalidSlot;
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        pti[j] = e[j] != kInvalidSlot ? e[j] + sparse_leaf_local(sub[j]) : kInvalidSlot;
                        slot[j] = e[j] != kInvalidSlot ? __ldg(P.vol.pt + pti[j]) : kInvalidSlot;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) slot[j] = __ldg(P.vol.pt + (j < nvalid ? pti[j] : 0u));
                }
                // (the entry at miss_at is selected in this loop: indexing the arrays with a run-time
                // index would move them to local memory)
                int miss_at = kBatch;
                uint32_t miss_pti = 0u;
#pragma unroll
                for (int j = kBatch - 1; j >= 0; --j)
                    if (j < nvalid && slot[j] == kInvalidSlot) {
                        miss_at = j;
                        miss_pti = pti[j];
                    }
                // usage stamps (one store per brick change)
#pragma unroll
                for (int j = 0; j < kBatch; ++j) {
                    if (j < nvalid && j < miss_at && pti[j] != cur_pti) {
                        cur_pti = pti[j];
                        if (P.last_used) P.last_used[slot[j]] = P.frame;
                    }
                }
                // ES: the value range and macro-cell span of the batch's last sample, loaded beside
                // the gathers and tested after compositing
                const bool test_last = ES && nvalid == kBatch && miss_at == kBatch;
                float2 rng_last = make_float2(0.f, 0.f);
                uint32_t span_last = 0u;
                if (test_last) {
                    rng_last = __ldg(P.vol.range + slot[kBatch - 1]);
                    span_last = __ldg(P.vol.cells + slot[kBatch - 1] * ncells + cell_last);
                }
                // (c) gathers, all issued together (unused samples read slot 0, element 0)
                float val[kBatch];
#pragma unroll
                for (int j = 0; j < kBatch; ++j) {
                    const bool use = j < nvalid && j < miss_at;
                    const unsigned long long base = use ? (unsigned long long)slot[j] * slot_stride + loc[j] : 0ull;
                    val[j] = sample_value<DT, BS, Q>(P.vol.atlas, base, B1, wgt[j]);
                }
                const int stop = min(nvalid, miss_at);
                bool fin = false;
                if constexpr (MODE != kMip) {
                    // TF rows: indices and weights of the batch first, then each sample's row is
                    // read while the one before it is composited (no branch before the read)
                    int ti[kBatch];
                    float tw[kBatch];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) tf_index<DT>(val[j], ti[j], tw[j]);
                    float4 an = s_tf[ti[0]], dn = s_tfd[ti[0]];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const float4 a = an, dab = dn;
                        if (j + 1 < kBatch) {
                            an = s_tf[ti[j + 1]];
                            dn = s_tfd[ti[j + 1]];
                        }
                        if (j < stop && !fin) {
                            if (GRAD && k > 0 && (k & ((1 << P.ckpt_shift) - 1)) == 0)
                                P.ckpt[(long long)((k >> P.ckpt_shift) - 1) * P.nrays + ray] = T;
                            if (GRAD && P.tape) {
                                // the sample's value, for the adjoint's recompute of T: staged in groups
                                // of 4 aligned samples, written 16 bytes at a time
                                tb = make_float4(tb.y, tb.z, tb.w, val[j]);
                                if ((k & 3) == 3) {
                                    if (k - 3 >= tb_from) {
                                        *reinterpret_cast<float4*>(P.tape + tape_at(P.nrays, ray, k - 3)) = tb;
                                    } else {  // the group began before this lane took the ray over
                                        if (k - 2 >= tb_from) P.tape[tape_at(P.nrays, ray, k - 2)] = tb.y;
                                        if (k - 1 >= tb_from) P.tape[tape_at(P.nrays, ray, k - 1)] = tb.z;
                                        P.tape[tape_at(P.nrays, ray, k)] = tb.w;
                                    }
                                }
                            }
                            fin = composite_row<MODE, LS>(tw[j], a, dab, amax_tf, et, T, C0, C1, C2,
                                                          LS ? lv[j] : 0);
                            ++k;
                            if (LS) tcur = tv[j + 1];
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        if (j < stop && !fin) {
                            fin = composite_sample<DT, MODE>(val[j], s_tf, s_tfd, amax_tf, et, T, C0, C1, C2);
                            ++k;
                        }
                    }
                }
                bool fell = false;
                if (!GRAD && P.preview && !fin && miss_at < kBatch) {
                    // preview (Sec. III-H): sample k lies in a brick that is not resident.  Request the
                    // brick for the refinement and take the sample on the finest coarser resident
                    // level (left out when none is).
                    if (SP) {
                        if (P.req_table64)
                            request_brick64(P, sparse_request_key<LOD>(tcur_or_t(LS, tcur, t0, k, step), o0, o1, o2, d0,
                                                                       d1, d2, lodscale, P.lod_bias, nlev, s_lv,
                                                                       bshift, bmask, row));
                    } else if (P.req_table && miss_pti != cur_pti) {
                        request_brick(P, miss_pti + 1u);
                    }
                    cur_pti = SP ? kInvalidSlot : miss_pti;
                    const float tk = LS ? tcur : __fadd_rn(t0, __fmul_rn((float)k, step));
                    const int lk = LOD ? lod_level(tk, lodscale, P.lod_bias, nlev) : 0;
                    const Fallback F = preview_fallback<LOD, SP>(P.vol.pt, tk, o0, o1, o2, d0, d1, d2, lodscale,
                                                                 P.lod_bias, nlev, s_lv, bshift, bmask, row);
                    if (F.ok) {
                        if (P.last_used) P.last_used[F.slot] = P.frame;
                        const float v = sample_value<DT, BS, Q>(
                            P.vol.atlas, (unsigned long long)F.slot * slot_stride + F.local, B1, F.w);
                        fin = composite_sample<DT, MODE, LS>(v, s_tf, s_tfd, amax_tf, et, T, C0, C1, C2, lk);
                    }
                    ++k;
                    if (LS) tcur = next_t_level_step(tk, step, lk);
                    fell = true;
                    const unsigned m = __activemask();
                    if ((int)lane == __ffs(m) - 1) atomicAdd(&P.counters[kPreview], (unsigned)__popc(m));
                }
                if (!fin && !fell && nvalid < kBatch && nvalid <= miss_at) fin = true;  // left the volume
                if (test_last && !fin) {
                    // sample k - 1 (the batch's last) lies in a brick or macro-cell that cannot change
                    // the state: the next batch starts at the block's end
                    sk_brick = brick_skippable<DT, MODE>(rng_last, s_apre, s_amx, T);
                    sk = sk_brick || span_skippable<MODE>(span_last, s_apre, s_amx, T);
                } else if (fin) {
                    const float4 bg = P.bg;
                    if (MODE == kMop || MODE == kMip) {
                        // the kept sample composited once over the background
                        float al = 0.0f;
                        if (MODE == kMop) {
                            al = T;
                        } else if (T >= 0.0f) {  // the TF at the largest coordinate
                            const int i = min((int)T, 254);
                            const float wt = T - (float)i;
                            const float4 a = s_tf[i], dab = s_tfd[i];
                            al = fmaf(wt, dab.w, a.w);
                            C0 = fmaf(wt, dab.x, a.x);
                            C1 = fmaf(wt, dab.y, a.y);
                            C2 = fmaf(wt, dab.z, a.z);
                        }
                        const float tb = 1.0f - al;
                        P.out[ray] = make_float4(fmaf(al, C0, tb * bg.x), fmaf(al, C1, tb * bg.y),
                                                 fmaf(al, C2, tb * bg.z), fmaf(tb, bg.w, al));
                    } else {
                        P.out[ray] = make_float4(fmaf(T, bg.x, C0), fmaf(T, bg.y, C1), fmaf(T, bg.z, C2),
                                                 fmaf(T, bg.w, 1.0f - T));
                    }
                    if (P.nsamp) P.nsamp[ray] = k;
                    if (GRAD) {
                        P.ray_n[ray] = k;
                        if (P.tape) tape_flush(P.tape, P.nrays, ray, k, tb_from, tb);
                    }
                    if (P.tile_cost && my_tile >= 0) atomicMax(&P.tile_cost[my_tile], k);
                    active = false;
                } else if (!fell && miss_at < kBatch) {
                    // wait for the missing brick: sample k (= the first missing one) resumes later
                    if (SP && P.req_table64) {
                        request_brick64(P, sparse_request_key<LOD>(__fadd_rn(t0, __fmul_rn((float)k, step)), o0, o1, o2,
                                                                   d0, d1, d2, lodscale, P.lod_bias, nlev, s_lv, bshift,
                                                                   bmask, row));
                        suspend_ray(P, ray, k, C0, C1, C2, T, 0.0f);
                    } else if (!SP && P.req_table) {
                        request_brick(P, miss_pti + 1u);
                        if (!LS && P.prefetch)
                            prefetch_next_brick<LOD>(P, k, miss_pti, o0, o1, o2, d0, d1, d2, t0, t1, lodscale, s_lv,
                                                     bshift, bmask, row, B1 - 1);
                        if (GRAD && P.tape) tape_flush(P.tape, P.nrays, ray, k, tb_from, tb);
                        suspend_ray(P, ray, k, C0, C1, C2, T, LS ? tcur : 0.0f);
                    } else {
                        atomicAdd(&P.counters[kDevError], 1u);
                    }
                    active = false;
                }
            }
            act = __ballot_sync(kFull, active);
        } while (__popc(act) >= thresh);
    }
}

}  // namespace
}  // namespace volrc
