// kernels_volume.cu -- brick upload/transcode with apron, LOD downsample, page-table update.
//
// Slot layouts (include/vol.h): compact slots hold the (B+1)^3 voxels of a brick and its
// +x/+y/+z apron; quad slots hold B x B x (B+1) entries of four voxels each, entry (x, y, z)
// = voxels (x, y), (x+1, y), (x, y+1), (x+1, y+1) of slice z of that region.
#include <algorithm>

#include "internal.cuh"

namespace volrc {
namespace {

// ---- storage conversions (normalised value -> stored type) ----
// u16 -> f16: binary16 (round to nearest even) of the binary32 quotient u / 65535.
template <int SRC, int DST>
struct Convert;
template <> struct Convert<VOL_U8, VOL_U8> {
    static __device__ __forceinline__ uint8_t run(uint8_t v) { return v; }
};
template <> struct Convert<VOL_U16, VOL_U16> {
    static __device__ __forceinline__ uint16_t run(uint16_t v) { return v; }
};
template <> struct Convert<VOL_F16, VOL_F16> {
    static __device__ __forceinline__ __half run(__half v) { return v; }
};
template <> struct Convert<VOL_F32, VOL_F32> {
    static __device__ __forceinline__ float run(float v) { return v; }
};
template <> struct Convert<VOL_U16, VOL_F16> {
    static __device__ __forceinline__ __half run(uint16_t v) { return __float2half_rn(__fdiv_rn((float)v, 65535.0f)); }
};
template <> struct Convert<VOL_U8, VOL_F32> {
    static __device__ __forceinline__ float run(uint8_t v) { return __fdiv_rn((float)v, 255.0f); }
};
template <> struct Convert<VOL_U16, VOL_F32> {
    static __device__ __forceinline__ float run(uint16_t v) { return __fdiv_rn((float)v, 65535.0f); }
};

template <int DT> struct Stored;
template <> struct Stored<VOL_U8> { using T = uint8_t; };
template <> struct Stored<VOL_U16> { using T = uint16_t; };
template <> struct Stored<VOL_F16> { using T = __half; };
template <> struct Stored<VOL_F32> { using T = float; };

// one quad entry written with a single vector store
template <int DT>
__device__ __forceinline__ void store4(typename Stored<DT>::T* p, typename Stored<DT>::T a, typename Stored<DT>::T b,
                                       typename Stored<DT>::T c, typename Stored<DT>::T d) {
    if constexpr (DT == VOL_U8) {
        *(uchar4*)p = make_uchar4(a, b, c, d);
    } else if constexpr (DT == VOL_U16) {
        *(ushort4*)p = make_ushort4(a, b, c, d);
    } else if constexpr (DT == VOL_F16) {
        *(ushort4*)p = make_ushort4(__half_as_ushort(a), __half_as_ushort(b), __half_as_ushort(c), __half_as_ushort(d));
    } else {
        *(float4*)p = make_float4(a, b, c, d);
    }
}

constexpr int kThreads = 256;

// One thread per slot voxel (compact) or entry (quad): grid.x covers the slot, grid.y/z bricks.
__device__ __forceinline__ long long brick_index() {
    return (long long)blockIdx.y + (long long)gridDim.y * blockIdx.z;
}

__device__ __forceinline__ int slot_items(const VolDev& vol) {
    const int B1 = vol.B1, B = B1 - 1;
    return vol.quad ? B * B * B1 : B1 * B1 * B1;
}

template <int SRC, int DST>
__global__ void __launch_bounds__(kThreads) k_upload_level(const typename Stored<SRC>::T* __restrict__ src,
                                                           typename Stored<DST>::T* __restrict__ atlas,
                                                           VolDev vol, int level,
                                                           const uint32_t* __restrict__ slots, long long nbricks) {
    const long long b = brick_index();
    if (b >= nbricks) return;
    const int B1 = vol.B1, B = B1 - 1;
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (r >= slot_items(vol)) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    const LevelDev& L = vol.lv[level];
    const int bx = (int)(b % L.nb[0]), by = (int)((b / L.nb[0]) % L.nb[1]), bz = (int)(b / ((long long)L.nb[0] * L.nb[1]));
    const long long sy = L.D[0], sz = (long long)L.D[0] * L.D[1];
    if (!vol.quad) {
        const int lx = r % B1, ly = (r / B1) % B1, lz = r / (B1 * B1);
        const long long gx = min(bx * B + lx, L.D[0] - 1), gy = min(by * B + ly, L.D[1] - 1), gz = min(bz * B + lz, L.D[2] - 1);
        atlas[(unsigned long long)slot * vol.slot_elems + r] = Convert<SRC, DST>::run(src[gx + gy * sy + gz * sz]);
        return;
    }
    const int lx = r % B, ly = (r / B) % B, lz = r / (B * B);
    const long long x0 = min(bx * B + lx, L.D[0] - 1), x1 = min(bx * B + lx + 1, L.D[0] - 1);
    const long long y0 = min(by * B + ly, L.D[1] - 1), y1 = min(by * B + ly + 1, L.D[1] - 1);
    const long long zo = (long long)min(bz * B + lz, L.D[2] - 1) * sz;
    store4<DST>(atlas + ((unsigned long long)slot * vol.slot_entries + r) * 4,
                Convert<SRC, DST>::run(src[x0 + y0 * sy + zo]), Convert<SRC, DST>::run(src[x1 + y0 * sy + zo]),
                Convert<SRC, DST>::run(src[x0 + y1 * sy + zo]), Convert<SRC, DST>::run(src[x1 + y1 * sy + zo]));
}

// n bricks of (B+1)^3 voxels each (compact, apron included), packed in src, into slots[i].
template <int SRC, int DST>
__global__ void __launch_bounds__(kThreads) k_upload_bricks(const typename Stored<SRC>::T* __restrict__ src,
                                                            typename Stored<DST>::T* __restrict__ atlas, VolDev vol,
                                                            const uint32_t* __restrict__ slots, long long n) {
    const long long b = brick_index();
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (b >= n || r >= slot_items(vol)) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    const int B1 = vol.B1, B = B1 - 1;
    const long long nvox = (long long)B1 * B1 * B1;
    const typename Stored<SRC>::T* s = src + b * nvox;
    if (!vol.quad) {
        atlas[(unsigned long long)slot * vol.slot_elems + r] = Convert<SRC, DST>::run(s[r]);
        return;
    }
    const int lx = r % B, ly = (r / B) % B, lz = r / (B * B);
    const int i = (lz * B1 + ly) * B1 + lx;
    store4<DST>(atlas + ((unsigned long long)slot * vol.slot_entries + r) * 4, Convert<SRC, DST>::run(s[i]),
                Convert<SRC, DST>::run(s[i + 1]), Convert<SRC, DST>::run(s[i + B1]), Convert<SRC, DST>::run(s[i + B1 + 1]));
}

// Voxel (cx, cy, cz) of a fine level, read through that level's page table (any layout).
// *bad is set when its brick is not resident.
template <int DT>
__device__ __forceinline__ typename Stored<DT>::T fine_voxel(const typename Stored<DT>::T* atlas, const VolDev& vol,
                                                             const LevelDev& F, int cx, int cy, int cz, bool* bad) {
    const uint32_t pti =
        F.pt_off + (uint32_t)((cx >> vol.bshift) + F.nb[0] * ((cy >> vol.bshift) + F.nb[1] * (cz >> vol.bshift)));
    const uint32_t cs = vol.pt[pti];
    if (cs == kInvalidSlot) {
        *bad = true;
        return typename Stored<DT>::T(0);
    }
    const int lx = cx & vol.bmask, ly = cy & vol.bmask, lz = cz & vol.bmask;
    if (vol.quad) {
        const int B = vol.B1 - 1;
        return atlas[((unsigned long long)cs * vol.slot_entries + (unsigned)((lz * B + ly) * B + lx)) * 4];
    }
    const int B1 = vol.B1;
    return atlas[(unsigned long long)cs * vol.slot_elems + (unsigned)((lz * B1 + ly) * B1 + lx)];
}

// Coarse voxel g of a level from the level below by the 2x2x2 box filter (Sec. III-D):
// children 2g and 2g+1 per axis, an index past the edge replaced by the last fine voxel;
// integer types (sum + 4) >> 3, float types a binary32 sum in (dz, dy, dx) order times 0.125.
template <int DT>
__device__ __forceinline__ typename Stored<DT>::T coarse_voxel(const typename Stored<DT>::T* atlas, const VolDev& vol,
                                                               const LevelDev& F, int gx, int gy, int gz, bool* bad) {
    using VT = typename Stored<DT>::T;
    int isum = 0;
    float fsum = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dz = c >> 2, dy = (c >> 1) & 1, dx = c & 1;
        const VT val = fine_voxel<DT>(atlas, vol, F, min(2 * gx + dx, F.D[0] - 1), min(2 * gy + dy, F.D[1] - 1),
                                      min(2 * gz + dz, F.D[2] - 1), bad);
        if constexpr (DT == VOL_U8 || DT == VOL_U16) isum += (int)val;
        else if constexpr (DT == VOL_F16) fsum = __fadd_rn(fsum, __half2float(val));
        else fsum = __fadd_rn(fsum, val);
    }
    if constexpr (DT == VOL_U8 || DT == VOL_U16) return (VT)((isum + 4) >> 3);
    else if constexpr (DT == VOL_F16) return __float2half_rn(__fmul_rn(fsum, 0.125f));
    else return __fmul_rn(fsum, 0.125f);
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_downsample(typename Stored<DT>::T* __restrict__ atlas, VolDev vol,
                                                         int level, const uint32_t* __restrict__ slots,
                                                         long long nbricks, unsigned* err) {
    const long long b = brick_index();
    if (b >= nbricks) return;
    const int B1 = vol.B1, B = B1 - 1;
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (r >= slot_items(vol)) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    const LevelDev& L = vol.lv[level];
    const LevelDev& F = vol.lv[level - 1];
    const int bx = (int)(b % L.nb[0]), by = (int)((b / L.nb[0]) % L.nb[1]), bz = (int)(b / ((long long)L.nb[0] * L.nb[1]));
    bool bad = false;
    if (!vol.quad) {
        const int lx = r % B1, ly = (r / B1) % B1, lz = r / (B1 * B1);
        const auto v = coarse_voxel<DT>(atlas, vol, F, min(bx * B + lx, L.D[0] - 1), min(by * B + ly, L.D[1] - 1),
                                        min(bz * B + lz, L.D[2] - 1), &bad);
        if (bad) {
            atomicAdd(err, 1u);
            return;
        }
        atlas[(unsigned long long)slot * vol.slot_elems + r] = v;
        return;
    }
    const int lx = r % B, ly = (r / B) % B, lz = r / (B * B);
    const int x0 = min(bx * B + lx, L.D[0] - 1), x1 = min(bx * B + lx + 1, L.D[0] - 1);
    const int y0 = min(by * B + ly, L.D[1] - 1), y1 = min(by * B + ly + 1, L.D[1] - 1);
    const int z = min(bz * B + lz, L.D[2] - 1);
    const auto v0 = coarse_voxel<DT>(atlas, vol, F, x0, y0, z, &bad);
    const auto v1 = coarse_voxel<DT>(atlas, vol, F, x1, y0, z, &bad);
    const auto v2 = coarse_voxel<DT>(atlas, vol, F, x0, y1, z, &bad);
    const auto v3 = coarse_voxel<DT>(atlas, vol, F, x1, y1, z, &bad);
    if (bad) {
        atomicAdd(err, 1u);
        return;
    }
    store4<DT>(atlas + ((unsigned long long)slot * vol.slot_entries + r) * 4, v0, v1, v2, v3);
}

// Transfer-function coordinate x = 255 clamp(v, 0, 1) of a stored value (u8: v; u16: v / 65535;
// floats: v), with the arithmetic the render kernels use.
template <int DT>
__device__ __forceinline__ float stored_coord(float v) {
    if (DT == VOL_U8) return v;
    if (DT == VOL_U16) return v * (255.0f / 65535.0f);
    return fminf(fmaxf(v, 0.0f), 1.0f) * 255.0f;
}

// Stored voxel (x, y, z), 0 <= x, y, z <= B, of slot a (either layout).
template <int DT>
__device__ __forceinline__ float slot_voxel(const typename Stored<DT>::T* a, bool quad, int B, int x, int y, int z) {
    long long i;
    if (quad) i = 4ll * (((long long)z * B + min(y, B - 1)) * B + min(x, B - 1)) + (x == B) + 2 * (y == B);
    else i = ((long long)z * (B + 1) + y) * (B + 1) + x;
    if constexpr (DT == VOL_F16) return __half2float(a[i]);
    else return (float)a[i];
}

// Value range of a slot (its brick plus apron, any layout): the render loop skips bricks whose
// range the transfer function maps to zero opacity.  And per macro-cell (local voxels
// [c M, c M + M] per axis: every corner a trilinear sample inside the cell reads) the span of TF
// entries [lo, hi] a lookup there can touch: the entries of the coordinates of the cell's
// smallest and largest value, widened by one entry on each side for the last-bit rounding of the
// interpolation (floats may overshoot their corners by an ulp).  A cell holding a NaN, or one
// whose range is not ordered, spans every entry.
template <int DT>
__global__ void __launch_bounds__(kThreads) k_slot_range(const typename Stored<DT>::T* __restrict__ atlas, VolDev vol,
                                                         float2* range, uint16_t* cells,
                                                         const uint32_t* __restrict__ slots) {
    __shared__ float s_lo[kThreads / 32], s_hi[kThreads / 32];
    const uint32_t slot = slots[blockIdx.x];
    if (slot == kInvalidSlot) return;
    const int B1 = vol.B1, B = B1 - 1;
    const long long n = vol.quad ? 4ll * B * B * B1 : (long long)B1 * B1 * B1;
    const typename Stored<DT>::T* a = atlas + (unsigned long long)slot * vol.slot_elems;
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        float v;
        if constexpr (DT == VOL_F16) v = __half2float(a[i]);
        else v = (float)a[i];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) {
            lo = fminf(lo, s_lo[w]);
            hi = fmaxf(hi, s_hi[w]);
        }
        range[slot] = make_float2(lo, hi);
    }
    if (!cells) return;
    const int cb = vol.cbits, M = 1 << vol.cshift, CB = 1 << cb;
    const int ncell = 1 << (3 * cb);
    const bool quad = vol.quad != 0;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int x0 = (c & (CB - 1)) * M, y0 = ((c >> cb) & (CB - 1)) * M, z0 = (c >> (2 * cb)) * M;
        float clo = __int_as_float(0x7f800000), chi = -__int_as_float(0x7f800000);
        bool nan = false;
        for (int z = z0; z <= z0 + M; ++z)
            for (int y = y0; y <= y0 + M; ++y)
                for (int x = x0; x <= x0 + M; ++x) {
                    const float v = slot_voxel<DT>(a, quad, B, x, y, z);
                    nan |= v != v;
                    clo = fminf(clo, v);
                    chi = fmaxf(chi, v);
                }
        uint16_t span = 0xFF00u;  // entries 0 .. 255
        if (!nan && clo <= chi) {
            const int ilo = max((int)stored_coord<DT>(clo) - 1, 0);
            const int ihi = min((int)stored_coord<DT>(chi) + 2, 255);
            span = (uint16_t)(ilo | (ihi << 8));
        }
        cells[(unsigned long long)slot * ncell + c] = span;
    }
}

// Adjoint of one box-filter level (k_downsample): fine voxel i has the single parent i >> 1 per
// axis, and along an axis of odd size the last fine voxel fills both child places of its
// parent (the filter replaces the missing child by it), so it takes 2 shares there.
__global__ void k_downsample_transpose(const float* __restrict__ coarse, float* __restrict__ fine, int Fx, int Fy,
                                       int Fz) {
    const long long n = (long long)Fx * Fy * Fz;
    const int Cx = (Fx + 1) / 2, Cy = (Fy + 1) / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Fx), y = (int)((i / Fx) % Fy), z = (int)(i / ((long long)Fx * Fy));
        const int m = ((Fx & 1) && x == Fx - 1 ? 2 : 1) * ((Fy & 1) && y == Fy - 1 ? 2 : 1) * ((Fz & 1) && z == Fz - 1 ? 2 : 1);
        const float g = coarse[(x >> 1) + (long long)Cx * ((y >> 1) + (long long)Cy * (z >> 1))];
        if (g != 0.0f) fine[i] += g * (0.125f * (float)m);
    }
}

__global__ void k_pt_update(uint32_t* pt, const uint32_t* idx, const uint32_t* val, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicExch(&pt[idx[i]], val[i]);
}

dim3 brick_grid(const VolDev& vol, long long nbricks) {
    const int B1 = vol.B1, B = B1 - 1;
    const int items = vol.quad ? B * B * B1 : B1 * B1 * B1;
    const unsigned gx = (unsigned)((items + kThreads - 1) / kThreads);
    const long long gy = nbricks < 65535 ? nbricks : 65535;
    const long long gz = (nbricks + gy - 1) / gy;
    return dim3(gx, (unsigned)(gy > 0 ? gy : 1), (unsigned)(gz > 0 ? gz : 1));
}

}  // namespace

cudaError_t launch_upload_level(int dst, int src_t, const void* src, const VolDev& vol, int level,
                                const uint32_t* slots, long long nbricks, cudaStream_t s) {
    if (nbricks <= 0) return cudaSuccess;
    const dim3 grid = brick_grid(vol, nbricks);
#define VOLRC_UP(S, D)                                                                                  \
    if (src_t == S && dst == D) {                                                                       \
        k_upload_level<S, D><<<grid, kThreads, 0, s>>>((const Stored<S>::T*)src, (Stored<D>::T*)vol.atlas, \
                                                       vol, level, slots, nbricks);                     \
        return cudaGetLastError();                                                                      \
    }
    VOLRC_UP(VOL_U8, VOL_U8)
    VOLRC_UP(VOL_U16, VOL_U16)
    VOLRC_UP(VOL_F16, VOL_F16)
    VOLRC_UP(VOL_F32, VOL_F32)
    VOLRC_UP(VOL_U16, VOL_F16)
    VOLRC_UP(VOL_U8, VOL_F32)
    VOLRC_UP(VOL_U16, VOL_F32)
#undef VOLRC_UP
    return cudaErrorInvalidValue;
}

cudaError_t launch_upload_bricks(int dst, int src_t, const void* src, const VolDev& vol, const uint32_t* slots,
                                 long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid = brick_grid(vol, n);
#define VOLRC_UPB(S, D)                                                                                      \
    if (src_t == S && dst == D) {                                                                            \
        k_upload_bricks<S, D><<<grid, kThreads, 0, s>>>((const Stored<S>::T*)src, (Stored<D>::T*)vol.atlas,  \
                                                        vol, slots, n);                                      \
        return cudaGetLastError();                                                                           \
    }
    VOLRC_UPB(VOL_U8, VOL_U8)
    VOLRC_UPB(VOL_U16, VOL_U16)
    VOLRC_UPB(VOL_F16, VOL_F16)
    VOLRC_UPB(VOL_F32, VOL_F32)
    VOLRC_UPB(VOL_U16, VOL_F16)
    VOLRC_UPB(VOL_U8, VOL_F32)
    VOLRC_UPB(VOL_U16, VOL_F32)
#undef VOLRC_UPB
    return cudaErrorInvalidValue;
}

cudaError_t launch_downsample(int dtype, const VolDev& vol, int level, const uint32_t* slots, long long nbricks,
                              unsigned* err, cudaStream_t s) {
    if (nbricks <= 0) return cudaSuccess;
    const dim3 grid = brick_grid(vol, nbricks);
    switch (dtype) {
    case VOL_U8: k_downsample<VOL_U8><<<grid, kThreads, 0, s>>>((uint8_t*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_U16: k_downsample<VOL_U16><<<grid, kThreads, 0, s>>>((uint16_t*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_F16: k_downsample<VOL_F16><<<grid, kThreads, 0, s>>>((__half*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_F32: k_downsample<VOL_F32><<<grid, kThreads, 0, s>>>((float*)vol.atlas, vol, level, slots, nbricks, err); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_slot_range(int dtype, const VolDev& vol, float2* range, uint16_t* cells, const uint32_t* slots,
                              long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    for (long long i0 = 0; i0 < n; i0 += 1ll << 30) {
        const unsigned g = (unsigned)((n - i0) < (1ll << 30) ? (n - i0) : (1ll << 30));
        switch (dtype) {
        case VOL_U8: k_slot_range<VOL_U8><<<g, kThreads, 0, s>>>((const uint8_t*)vol.atlas, vol, range, cells, slots + i0); break;
        case VOL_U16: k_slot_range<VOL_U16><<<g, kThreads, 0, s>>>((const uint16_t*)vol.atlas, vol, range, cells, slots + i0); break;
        case VOL_F16: k_slot_range<VOL_F16><<<g, kThreads, 0, s>>>((const __half*)vol.atlas, vol, range, cells, slots + i0); break;
        case VOL_F32: k_slot_range<VOL_F32><<<g, kThreads, 0, s>>>((const float*)vol.atlas, vol, range, cells, slots + i0); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_downsample_transpose(const float* coarse, float* fine, const int Dfine[3], cudaStream_t s) {
    const long long n = (long long)Dfine[0] * Dfine[1] * Dfine[2];
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 65536);
    k_downsample_transpose<<<(unsigned)blocks, 256, 0, s>>>(coarse, fine, Dfine[0], Dfine[1], Dfine[2]);
    return cudaGetLastError();
}

cudaError_t launch_pt_update(uint32_t* pt, const uint32_t* idx, const uint32_t* val, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_pt_update<<<(n + 255) / 256, 256, 0, s>>>(pt, idx, val, n);
    return cudaGetLastError();
}

}  // namespace volrc
