// internal.cuh -- device-side structures shared by the runtime and the kernels.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vol.h"

namespace volrc {

constexpr uint32_t kInvalidSlot = 0xFFFFFFFFu;
constexpr int kMaxLevels = VOL_MAX_LEVELS;
constexpr int kCkptEvery = 32;      // transmittance checkpoint spacing (samples), the largest allowed
constexpr int kCkptShift = 5;       // log2 kCkptEvery
// Macro-cells for empty-space skipping: cubes of 2^kCellShift voxels (at most 8 per brick axis;
// a brick of 2^kCellShift voxels or fewer per axis is one cell).  Measured on the 1024^3 and
// 2048^3 frames: 8-voxel cells beat 4-voxel ones (2048^3, 32^3 bricks: 52.8 against 54.1 ms),
// 16-voxel ones skip half as many emission/absorption samples of the noise volume.
#ifndef VOLRC_CELL_SHIFT
#define VOLRC_CELL_SHIFT 3
#endif
constexpr int kCellShift = VOLRC_CELL_SHIFT;
// log2 of the macro-cells per axis of a brick of 2^bshift voxels per axis
__host__ __device__ constexpr int cell_bits_for(int bshift) {
    return bshift - kCellShift < 0 ? 0 : (bshift - kCellShift > 3 ? 3 : bshift - kCellShift);
}
// Sample indices of a ray stay below this, so that they and small offsets of them are exact in
// binary32 (past 2^24, neighbouring indices round to the same depth).
constexpr double kMaxSamplesPerRay = 16777216.0 - 64.0;
constexpr int kRenderThreads = 128; // threads per CTA of the render kernels
constexpr int kMaxProbe = 64;       // bounded linear probing of the request table
#ifndef VOLRC_PREFETCH_BRICKS
#define VOLRC_PREFETCH_BRICKS 8
#endif
constexpr int kPrefetchBricks = VOLRC_PREFETCH_BRICKS;  // look-ahead of a waiting ray, in bricks

// Compositing variants of the forward kernel (template argument MODE of k_render).
constexpr int kDvr = 0;      // emission/absorption, front to back (Sec. IV-A)
constexpr int kDvrGrad = 1;  // the same, keeping transmittance checkpoints for the adjoint
constexpr int kMop = 2;      // maximum-opacity projection (Sec. V-A, Table I)
constexpr int kMip = 3;      // maximum-intensity projection

// Counter words of one render (device memory, reset before each pass).
enum Counter : int {
    kWork = 0,       // next work item (tile or suspended-ray chunk)
    kReqCount = 1,   // entries appended to the request list
    kSuspCount = 2,  // rays suspended in this pass
    kReqOverflow = 3,
    kDevError = 4,
    kPreview = 5,    // preview: samples taken from a coarser level, or left out
    kSkipped = 6,    // words 6-7: 64-bit count of samples jumped over by empty-space skipping
    kNumCounters = 8
};

struct LevelDev {
    int D[3];        // voxels per axis
    int nb[3];       // bricks per axis
    float r[3];      // D_l / D_0 per axis, binary32
    float ir[3];     // D_0 / D_l per axis (for estimates only; never in a decision)
    uint32_t pt_off; // first page-table entry (sparse table: of the level's top grid)
    int tn[3];       // sparse table: top-grid entries per axis, ceil(nb / 256)
};

// Sparse page table: a dense top grid per level (one entry per 256^3 bricks) -> middle page
// (16^3 entries) -> leaf page (16^3 entries, the slots).  Entries of the top grid and of
// middle pages hold the pool index of the child page's first entry, or kInvalidSlot.
constexpr int kPageShift = 4;  // 16 entries per axis and page
constexpr int kPageEntries = 1 << (3 * kPageShift);

struct ViewDev {
    float eye[3], right[3], up[3], fwd[3];
    float tan;        // tan_half_fov
    float tan_aspect; // tan_half_fov * aspect (binary32)
    float lodscale;   // (2 * tan_half_fov) / h (binary32)
    int w, h;
    int tiles_x;
    int tile_off;     // first work item of this view
    long long ray_off;// first ray (pixel) of this view in the packed image
    // pixels outside [cx0, cx1] x [cy0, cy1] miss the volume (a conservative bound of its
    // projection, with a margin; the whole image when no bound applies)
    int cx0, cx1, cy0, cy1;
};

struct SuspRec {       // a ray waiting for a brick
    long long ray;     // packed pixel index
    int k;             // next sample
    int tk_bits;       // level-scaled sampling: depth of sample k (float bits)
    float C[3], T;     // partial colour and transmittance
};

struct VolDev {
    const void* atlas;
    unsigned long long slot_elems; // voxels of storage per slot (padded)
    unsigned long long slot_entries; // quad layout: 4-voxel entries per slot (slot_elems / 4)
    int quad;                      // 1: quad layout, 0: compact (B+1)^3
    int bshift, bmask, B1;         // log2 B, B - 1, B + 1
    int nlevels;
    const uint32_t* pt;            // flat page table, or the sparse table's pool
    int sparse;                    // 1: three-level sparse page table
    const float2* range;           // per slot: min and max stored value (stored units)
    // per slot: the TF-entry span of each macro-cell (8 x 8 x 8 cells per brick, or B per axis
    // when B < 8; cell c covers local voxels [c M, c M + M] per axis, M = B >> cbits): byte 0 the
    // lowest and byte 1 the highest TF entry a trilinear lookup inside the cell can touch
    const uint16_t* cells;
    int cshift;                    // log2 M: a voxel's cell along an axis is (i0 & bmask) >> cshift
    int cbits;                     // log2 of the cells per brick axis
    LevelDev lv[kMaxLevels];
    float D0f[3];
};

struct RenderDev {
    VolDev vol;
    const ViewDev* views;
    int nviews;
    int nwork;          // tiles (fresh pass) or 32-ray chunks (resume pass)
    int resume;         // 0: fresh pass over tiles; 1: resume suspended rays
    int tile_w, tile_h;
    int refill_thresh;  // refill lanes when fewer than this many are active
    const float4* tf;
    float step, et;
    float4 bg;
    int lod_mode, lod_bias;
    int skip_empty;     // empty-space skipping: launch the ES variant of the kernel
    int preview;        // a sample on a non-resident brick uses the finest coarser resident level
    int level_step;     // level-scaled sampling (chooses the kernel variant)
    int prefetch;       // a suspended ray also requests this many bricks after the missing one
    float4* out;
    int* nsamp;
    unsigned* counters;
    // misses
    const SuspRec* susp_in;
    int nsusp_in;
    SuspRec* susp_out;
    unsigned* req_table;
    unsigned req_cap_mask;
    unsigned* req_list;
    unsigned req_list_cap;
    unsigned long long* req_table64;  // sparse page table: requests keyed by (level, brick)
    unsigned long long* req_list64;
    unsigned* last_used;
    unsigned frame;
    // gradient checkpoints: T before samples 2^ckpt_shift, 2 * 2^ckpt_shift, ... (ckpt_shift 5:
    // every 32nd sample; 0: every sample, the store-all debug mode)
    float* ckpt;
    long long nrays;
    int ckpt_shift;
    int* ray_n;
    // value tape (NULL: none): the interpolated value of sample k of a ray at
    // [(k / 32) * nrays + ray] * 32 + k % 32, for the adjoint's transmittance recompute
    float* tape;
    // scheduling: work item i of a fresh pass renders tile tile_order[i] (NULL: tile i);
    // every finished ray raises tile_cost[its tile] to its sample count: the tile's longest ray
    // (NULL: not recorded)
    const int* tile_order;
    int* tile_cost;
};

struct BackwardDev {
    VolDev vol;
    const ViewDev* views;
    int nviews;
    int nwork;          // work items: 32-ray parts of the tiles
    int tile_w, tile_h;
    const float4* tf;
    float step;
    float4 bg;
    const float4* drgba;
    float* dtf;
    float* dvox;                // level-0 gradient (NULL: none)
    float* dlev[kMaxLevels];    // gradient of each level's voxels; dlev[0] = dvox
    int lod_mode, lod_bias;
    unsigned* counters;
    const float* ckpt;
    int ckpt_shift;         // checkpoint spacing 2^ckpt_shift samples (0..kCkptShift)
    const float* tape;      // the forward's sample values (RenderDev::tape layout), or NULL
    long long nrays;
    const int* ray_n;
    const int* tile_order;  // longest-ray-first order of the tiles (NULL: tile i)
};

struct TraceDev {
    VolDev vol;
    ViewDev view;
    float step;
    int lod_mode, lod_bias;
    int level_step;     // samples dt * 2^l apart (level-scaled sampling)
    const int* pixels;
    int npix;
    int max_samples;
    vol_trace_rec* out;
    int* counts;
};

// ---- launchers (kernels_render.cu) ----
// mode: kDvr, kDvrGrad, kMop or kMip.
cudaError_t launch_render(int dtype, int mode, const RenderDev& p, int grid, cudaStream_t s);
cudaError_t launch_backward(int dtype, const BackwardDev& p, int grid, cudaStream_t s);
cudaError_t launch_trace(const TraceDev& p, cudaStream_t s);
int render_blocks_per_sm(int dtype, bool grad);
// Maximum projections (kernels_project.cu): the k_render variant for mode kMop or kMip.
const void* pick_render_projection(int dtype, int brick, bool quad, bool lod, int mode);
// Level-scaled sampling (kernels_lstep.cu): the emission/absorption variant.
const void* pick_render_level_step(int dtype, int brick, bool quad, bool lod);
// Sparse page table (kernels_sparse.cu): the emission/absorption variant.
const void* pick_render_sparse(int dtype, int brick, bool quad, bool lod);
// Empty-space skipping (kernels_skip.cu: emission/absorption; kernels_skip_project.cu: MOP, MIP):
// the variant for mode kDvr, kMop or kMip (nullptr for a quad layout with bricks other than 32 or 64).
const void* pick_render_skip(int dtype, int brick, bool quad, bool lod, int mode);
const void* pick_render_skip_projection(int dtype, int brick, bool quad, bool lod, int mode);
// order[] = tiles sorted by descending log2 bucket of cost[] (longest ray first); zeroes cost[].
// buckets: 64 ints of device scratch.
cudaError_t launch_tile_order(int* cost, int* order, int ntiles, int* buckets, cudaStream_t s);
int backward_blocks_per_sm(int dtype, bool lod, bool tape);

// ---- launchers (kernels_volume.cu) ----
// Write every brick of a dense level (src of src_dtype) into atlas slots.
cudaError_t launch_upload_level(int dst_dtype, int src_dtype, const void* src, const VolDev& vol,
                                int level, const uint32_t* slots_of_bricks, long long nbricks,
                                cudaStream_t s);
// Write n packed (B+1)^3 bricks (src of src_dtype, device) into slots[i] (device array).
cudaError_t launch_upload_bricks(int dst_dtype, int src_dtype, const void* src, const VolDev& vol,
                                 const uint32_t* slots, long long n, cudaStream_t s);
// Build level `level` (all bricks; slots_of_bricks indexed by brick id) from level-1.
cudaError_t launch_downsample(int dtype, const VolDev& vol, int level, const uint32_t* slots_of_bricks,
                              long long nbricks, unsigned* err, cudaStream_t s);
// Adjoint of one box-filter level: fine[i] += coarse[parent(i)] * (shares of i) / 8, for the
// level of dims Dfine filtered into the level of coarse (a child index past the edge counts as
// the last voxel, as in the filter).
cudaError_t launch_downsample_transpose(const float* coarse, float* fine, const int Dfine[3], cudaStream_t s);
// range[slots[i]] = (min, max) of the stored values of each listed slot, and the slot's macro-cell
// TF-entry spans in cells (one CTA per slot).
cudaError_t launch_slot_range(int dtype, const VolDev& vol, float2* range, uint16_t* cells, const uint32_t* slots,
                              long long n, cudaStream_t s);
// pt[idx[i]] = val[i] for i < n (atomic exchange; Sec. III-E parallel insert/remove).
cudaError_t launch_pt_update(uint32_t* pt, const uint32_t* idx, const uint32_t* val, int n,
                             cudaStream_t s);

}  // namespace volrc
