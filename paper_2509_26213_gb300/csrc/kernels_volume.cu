// kernels_volume.cu -- brick upload/transcode with apron, LOD downsample, page-table update.
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

constexpr int kThreads = 256;

// One thread per slot voxel (apron included): grid.x covers (B+1)^3, grid.y/z the bricks.
__device__ __forceinline__ long long brick_index() {
    return (long long)blockIdx.y + (long long)gridDim.y * blockIdx.z;
}

template <int SRC, int DST>
__global__ void __launch_bounds__(kThreads) k_upload_level(const typename Stored<SRC>::T* __restrict__ src,
                                                           typename Stored<DST>::T* __restrict__ atlas,
                                                           VolDev vol, int level,
                                                           const uint32_t* __restrict__ slots, long long nbricks) {
    const long long b = brick_index();
    if (b >= nbricks) return;
    const int B1 = vol.B1, B = B1 - 1;
    const int nvox = B1 * B1 * B1;
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (r >= nvox) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    const LevelDev& L = vol.lv[level];
    const int lx = r % B1, ly = (r / B1) % B1, lz = r / (B1 * B1);
    const int bx = (int)(b % L.nb[0]), by = (int)((b / L.nb[0]) % L.nb[1]), bz = (int)(b / ((long long)L.nb[0] * L.nb[1]));
    const int gx = min(bx * B + lx, L.D[0] - 1), gy = min(by * B + ly, L.D[1] - 1), gz = min(bz * B + lz, L.D[2] - 1);
    const long long si = (long long)gx + (long long)L.D[0] * ((long long)gy + (long long)L.D[1] * gz);
    atlas[(unsigned long long)slot * vol.slot_elems + r] = Convert<SRC, DST>::run(src[si]);
}

// n bricks of (B+1)^3 voxels each, packed in src, into slots[i].
template <int SRC, int DST>
__global__ void __launch_bounds__(kThreads) k_upload_bricks(const typename Stored<SRC>::T* __restrict__ src,
                                                            typename Stored<DST>::T* __restrict__ atlas,
                                                            unsigned long long slot_elems, int nvox,
                                                            const uint32_t* __restrict__ slots, long long n) {
    const long long b = brick_index();
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (b >= n || r >= nvox) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    atlas[(unsigned long long)slot * slot_elems + r] = Convert<SRC, DST>::run(src[b * nvox + r]);
}

// 2x2x2 box filter from level-1 into the slots of `level` (Sec. III-D).  Children are read
// through the fine level's page table; a child index past the edge is replaced by the last
// fine voxel.  Integer: (sum + 4) >> 3.  Float: binary32 sum in (dz, dy, dx) order, * 0.125.
template <int DT>
__global__ void __launch_bounds__(kThreads) k_downsample(typename Stored<DT>::T* __restrict__ atlas, VolDev vol,
                                                         int level, const uint32_t* __restrict__ slots,
                                                         long long nbricks, unsigned* err) {
    using VT = typename Stored<DT>::T;
    const long long b = brick_index();
    if (b >= nbricks) return;
    const int B1 = vol.B1, B = B1 - 1;
    const int nvox = B1 * B1 * B1;
    const int r = blockIdx.x * kThreads + threadIdx.x;
    if (r >= nvox) return;
    const uint32_t slot = slots[b];
    if (slot == kInvalidSlot) return;
    const LevelDev& L = vol.lv[level];
    const LevelDev& F = vol.lv[level - 1];
    const int lx = r % B1, ly = (r / B1) % B1, lz = r / (B1 * B1);
    const int bx = (int)(b % L.nb[0]), by = (int)((b / L.nb[0]) % L.nb[1]), bz = (int)(b / ((long long)L.nb[0] * L.nb[1]));
    const int g[3] = {min(bx * B + lx, L.D[0] - 1), min(by * B + ly, L.D[1] - 1), min(bz * B + lz, L.D[2] - 1)};
    int isum = 0;
    float fsum = 0.0f;
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dz = c >> 2, dy = (c >> 1) & 1, dx = c & 1;
        const int cx = min(2 * g[0] + dx, F.D[0] - 1), cy = min(2 * g[1] + dy, F.D[1] - 1), cz = min(2 * g[2] + dz, F.D[2] - 1);
        const uint32_t pti = F.pt_off + (uint32_t)((cx >> vol.bshift) + F.nb[0] * ((cy >> vol.bshift) + F.nb[1] * (cz >> vol.bshift)));
        const uint32_t cs = vol.pt[pti];
        if (cs == kInvalidSlot) {
            bad = true;
            continue;
        }
        const int lo = ((cz & vol.bmask) * B1 + (cy & vol.bmask)) * B1 + (cx & vol.bmask);
        const VT val = atlas[(unsigned long long)cs * vol.slot_elems + lo];
        if constexpr (DT == VOL_U8 || DT == VOL_U16) isum += (int)val;
        else if constexpr (DT == VOL_F16) fsum = __fadd_rn(fsum, __half2float(val));
        else fsum = __fadd_rn(fsum, val);
    }
    if (bad) {
        atomicAdd(err, 1u);
        return;
    }
    VT out;
    if constexpr (DT == VOL_U8 || DT == VOL_U16) out = (VT)((isum + 4) >> 3);
    else if constexpr (DT == VOL_F16) out = __float2half_rn(__fmul_rn(fsum, 0.125f));
    else out = __fmul_rn(fsum, 0.125f);
    atlas[(unsigned long long)slot * vol.slot_elems + r] = out;
}

__global__ void k_pt_update(uint32_t* pt, const uint32_t* idx, const uint32_t* val, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicExch(&pt[idx[i]], val[i]);
}

dim3 brick_grid(int nvox, long long nbricks) {
    const unsigned gx = (unsigned)((nvox + kThreads - 1) / kThreads);
    const long long gy = nbricks < 65535 ? nbricks : 65535;
    const long long gz = (nbricks + gy - 1) / gy;
    return dim3(gx, (unsigned)(gy > 0 ? gy : 1), (unsigned)(gz > 0 ? gz : 1));
}

}  // namespace

cudaError_t launch_upload_level(int dst, int src_t, const void* src, const VolDev& vol, int level,
                                const uint32_t* slots, long long nbricks, cudaStream_t s) {
    if (nbricks <= 0) return cudaSuccess;
    const int nvox = vol.B1 * vol.B1 * vol.B1;
    const dim3 grid = brick_grid(nvox, nbricks);
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
    const int nvox = vol.B1 * vol.B1 * vol.B1;
    const dim3 grid = brick_grid(nvox, n);
#define VOLRC_UPB(S, D)                                                                                     \
    if (src_t == S && dst == D) {                                                                           \
        k_upload_bricks<S, D><<<grid, kThreads, 0, s>>>((const Stored<S>::T*)src, (Stored<D>::T*)vol.atlas, \
                                                        vol.slot_elems, nvox, slots, n);                    \
        return cudaGetLastError();                                                                          \
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
    const int nvox = vol.B1 * vol.B1 * vol.B1;
    const dim3 grid = brick_grid(nvox, nbricks);
    switch (dtype) {
    case VOL_U8: k_downsample<VOL_U8><<<grid, kThreads, 0, s>>>((uint8_t*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_U16: k_downsample<VOL_U16><<<grid, kThreads, 0, s>>>((uint16_t*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_F16: k_downsample<VOL_F16><<<grid, kThreads, 0, s>>>((__half*)vol.atlas, vol, level, slots, nbricks, err); break;
    case VOL_F32: k_downsample<VOL_F32><<<grid, kThreads, 0, s>>>((float*)vol.atlas, vol, level, slots, nbricks, err); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pt_update(uint32_t* pt, const uint32_t* idx, const uint32_t* val, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_pt_update<<<(n + 255) / 256, 256, 0, s>>>(pt, idx, val, n);
    return cudaGetLastError();
}

}  // namespace volrc
