/*
 * vol.h -- C ABI of the GB300 bricked multi-resolution volume raycaster.
 *
 * The library renders a volume that is split into bricks (Drees & Risse,
 * "Palace", arXiv 2509.26213, Sec. III-A: h = floor(g / C), l = g mod C),
 * kept as a level-of-detail pyramid (Sec. III-D) whose resident bricks sit in
 * one device "atlas" and are found through one page table per level
 * (Sec. III-E).  Rendering is direct volume rendering (Sec. IV-A) with a 1D
 * RGBA transfer function (Fig. 1), footprint-based LOD selection (Sec. V-C),
 * early ray termination, and a brick-request queue for bricks that are not
 * resident (Sec. III-H).  An adjoint pass gives gradients with respect to the
 * transfer function and the level-0 voxels (not in the paper).
 *
 * Conventions shared by every entry point
 *   - Return value: VOL_OK (0) or a negative VOL_ERR_* code.  The message of
 *     the last failure on a volume is available from vol_last_error().
 *   - Coordinates: level-0 voxel units; the volume occupies [0, D) per axis
 *     and voxel i has its centre at i + 0.5.  Level l has D_l = ceil(D_{l-1}/2)
 *     voxels per axis and spacing D_0 / D_l (uniform physical size).
 *   - Dense voxel arrays are x fastest: index = x + Dx * (y + Dy * z).
 *   - Images are packed per view, row-major, y down: float RGBA [h][w][4].
 *   - Ownership: the caller owns every pointer it passes; the library never
 *     frees them and keeps none after the call returns, except that
 *     vol_render_backward() and vol_render_resume() use the buffers of the
 *     preceding vol_render() on the same volume.
 *   - Streams: all device work of a volume is ordered on the CUDA stream given
 *     to vol_create() / vol_set_stream() (NULL = the legacy default stream).
 *     Calls return once the work is enqueued, except where noted.
 *   - One volume is used by one host thread at a time.
 */
#ifndef VOLRC_VOL_H
#define VOLRC_VOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VOL_OK 0
#define VOL_ERR_INVALID_ARG (-1)      /* bad size, pointer, level, brick or parameter */
#define VOL_ERR_OOM (-2)              /* a device or pinned host allocation failed */
#define VOL_ERR_INCOMPLETE (-3)       /* rays are still waiting for non-resident bricks */
#define VOL_ERR_PROVIDER (-4)         /* the brick provider callback returned non-zero */
#define VOL_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define VOL_ERR_NO_FORWARD_STATE (-6) /* backward/resume without a matching render */
#define VOL_ERR_UNSUPPORTED (-7)      /* valid request outside what this build supports */
#define VOL_ERR_DEVICE (-8)           /* a device-side check failed (recorded, not trapped) */
#define VOL_ERR_CACHE_FULL (-9)       /* no brick slot could be freed */

#define VOL_MAX_LEVELS 16
#define VOL_MAX_VIEWS 1024

/* Storage type of the voxels in the atlas; values are normalised to [0, 1]
 * as u8 / 255, u16 / 65535, and floats as stored (clamped to [0, 1] before
 * the transfer function). */
typedef enum { VOL_U8 = 0, VOL_U16 = 1, VOL_F16 = 2, VOL_F32 = 3 } vol_dtype;

typedef struct vol_s *vol_t;

/* Pinhole camera.  For pixel (px, py) of a w x h image:
 *   u = ((px + 0.5) / w) * 2 - 1,  v = 1 - ((py + 0.5) / h) * 2,
 *   d = normalise(fwd + (u * tan_half_fov * aspect) * right + (v * tan_half_fov) * up)
 * in binary32 without contraction; the ray starts at eye (Fig. 1's
 * CameraState / entry_exit_points). */
typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float tan_half_fov; /* tan(vertical field of view / 2); must be > 0 and finite */
    float aspect;       /* w / h */
    int32_t w, h;
} vol_camera;

#define VOL_RENDER_GRAD 1u /* keep transmittance checkpoints for vol_render_backward */
/* Empty-space skipping (the paper's skipping of uniform chunks, Sec. III-H and Sec. IV-A):
 * after each batch of samples a ray tests the brick, and the macro-cell of 8^3 voxels inside
 * it, of its last sample; when the transfer function maps the block's stored value range to
 * zero opacity, the ray jumps to the block's last sample.  Those samples would composite
 * nothing (alpha exactly 0), so the image and the per-pixel sample counts are identical with
 * or without it; vol_stats.skipped_samples counts them.  (Emission/absorption, MOP and MIP on
 * the flat page table with uniform steps; other renders ignore the flag, and so does a quad
 * layout with bricks other than 32^3 or 64^3.) */
#define VOL_RENDER_SKIP_EMPTY 2u
/* With a batch provider, vol_render overlaps brick loading with rendering: while a pass
 * runs, the requests it appends are read and a library thread runs the provider on chunks
 * of them (one call at a time, from that thread) into a pinned host ring, from which queued
 * kernels upload the bricks after the pass; the next pass resumes the rays.  This flag
 * loads all requested bricks between passes instead, on the calling thread.  The image is
 * the same either way. */
#define VOL_RENDER_SERIAL_LOADS 4u
/* Progressive preview (Sec. III-H: a low-resolution image from coarser levels first, refined as
 * bricks arrive).  One pass: a sample whose brick on its level is not resident is taken on the
 * finest coarser level whose brick at that position is resident (left out when none is) instead
 * of waiting, and the brick it wanted is requested.  With a provider the requested bricks start
 * loading before the call returns (with a batch provider, overlapped with the pass; the chunk
 * still in generation is published by the next call), so repeated preview renders refine the
 * image; vol_stats.preview_samples counts the samples not on their own level (0: the image is
 * the full render's).  Not with VOL_RENDER_GRAD. */
#define VOL_RENDER_PREVIEW 8u
/* Level-scaled sampling (emission/absorption, no gradients): a sample on LOD level l stands
 * for 2^l reference steps.  t_0 = t0, t_{k+1} = t_k + step * 2^{l_k} (binary32), and the
 * sample's opacity is corrected to the longer step, a' = 1 - (1 - a)^(2^l), so a constant
 * medium keeps its transmittance while coarse levels take fewer samples.  Empty-space
 * skipping is not applied in this mode. */
#define VOL_RENDER_LEVEL_STEP 16u
/* With a provider, a ray that waits for a missing brick also requests the next bricks along it
 * (a look-ahead of eight bricks), so that it does not wait a round for each when it resumes; the
 * extra bricks may go unused.  This flag turns the look-ahead off.  Images do not change. */
#define VOL_RENDER_NO_PREFETCH 32u
/* Debug, with VOL_RENDER_GRAD only: keep the transmittance before every sample instead of every
 * 32nd (4 bytes per sample of each ray), so vol_render_backward() reads every T_k instead of
 * recomputing it forward within a 32-sample segment.  The gradients equal the checkpointed ones
 * up to the order of the atomic additions; it exists to test that recompute. */
#define VOL_RENDER_CKPT_ALL 64u
/* With VOL_RENDER_GRAD: the render keeps every sample's interpolated value (4 bytes per sample,
 * room for the longest ray's samples for every ray), and vol_render_backward() recomputes the
 * transmittance of a segment from its checkpoint and these values instead of interpolating
 * them again from the bricks; the gradients are the same.  This flag turns the value tape off
 * (the adjoint then interpolates again; it is also off when its memory cannot be allocated, and
 * with VOL_RENDER_CKPT_ALL). */
#define VOL_RENDER_GRAD_RECOMPUTE 128u

/* Compositing (vol_params.composite).
 * VOL_COMPOSITE_DVR: front-to-back emission/absorption with early termination (Sec. IV-A).
 * VOL_COMPOSITE_MOP: maximum-opacity projection, the mode of the paper's Kidney renderings
 *   (Sec. V-A, Table I): every sample is visited and the first one of largest TF opacity is
 *   kept (a later one replaces it only when strictly more opaque).  The ray stops early once
 *   the kept opacity reaches the largest opacity of any TF entry.
 * VOL_COMPOSITE_MIP: maximum-intensity projection: the largest TF coordinate
 *   x = 255 clamp(v, 0, 1) over the samples is kept and the TF looked up there.  The ray
 *   stops early at x = 255.
 * Both projections composite the kept (rgb, a) once over the background:
 *   out_rgb = a rgb + (1 - a) bg_rgb,  out_a = a + (1 - a) bg_a,
 * and give bg for a ray that misses the box.  With VOL_RENDER_SKIP_EMPTY, a ray skips a
 * brick or macro-cell whose stored value range bounds every sample's opacity (MOP) or
 * coordinate (MIP) at or below the kept one; the image does not change.  Neither has an
 * adjoint. */
#define VOL_COMPOSITE_DVR 0
#define VOL_COMPOSITE_MOP 1
#define VOL_COMPOSITE_MIP 2

typedef struct {
    float step;          /* sample spacing in level-0 voxels (> 0; at most 2^24 - 64 samples
                            along the volume diagonal, else VOL_ERR_INVALID_ARG) */
    float et_threshold;  /* stop a ray after the sample where 1 - T >= et_threshold */
    float bg[4];         /* background RGBA composited behind the volume */
    int32_t lod_mode;    /* 0: all samples on level 0; 1: footprint LOD (Sec. V-C) */
    int32_t lod_bias;    /* added to the footprint level before clamping to [0, L-1] */
    int32_t tile_w;      /* ray tile (work item) width in pixels; 0 = default 4 */
    int32_t tile_h;      /* ray tile height (tile_w * tile_h <= 4096); 0 = 8 */
    int32_t max_passes;  /* miss/refill passes per render when a provider is set; 0 = 256 */
    uint32_t flags;      /* VOL_RENDER_* bits */
    int32_t refill;      /* a warp fetches new rays once fewer lanes than this are busy
                            (1..32; 0 = default: 20 for emission/absorption, 28 for MOP and
                            MIP); performance only, never the image */
    int32_t ctas_per_sm; /* persistent CTAs per SM (0 = as many as fit) */
    int32_t composite;   /* VOL_COMPOSITE_* (0 = emission/absorption) */
} vol_params;

/* Atlas slot layouts (vol_plan / vol_create flags).
 * Default, "quad": a slot holds B x B x (B+1) entries, entry (x, y, z) being the
 * four voxels (x, y), (x+1, y), (x, y+1), (x+1, y+1) of slice z of the brick's
 * apron-extended region, stored together (4, 8, 8 or 16 bytes for u8, u16,
 * f16, f32), so the eight corners of a trilinear sample are two aligned loads.
 * It takes about 4x the memory of the voxels.
 * VOL_LAYOUT_COMPACT: a slot holds the (B+1)^3 voxels of the brick and its
 * +x/+y/+z apron; a sample reads eight scalars.  Both give identical images. */
#define VOL_LAYOUT_COMPACT 1u
/* Sparse page table (the paper's three-level page table, Sec. III-E and Sec. V-C's virtual
 * zettabyte volume): instead of one entry per brick of every level, each level has a dense top
 * grid with one entry per 256^3 bricks, pointing to a middle page (16^3 entries, one per 16^3
 * bricks), pointing to a leaf page (16^3 entries: the slots); pages are allocated as bricks
 * arrive and are never freed.  The volume may then hold more bricks than 32-bit indices can
 * count (up to 2^20 bricks per axis and level), e.g. a virtual volume whose bricks a
 * provider generates.  Needs cache_bytes > 0.  Bricks arrive through vol_upload_brick or a
 * provider (vol_upload_level and vol_build_lod are not available), brick loads are serial,
 * and rendering is emission/absorption without gradients, level-scaled sampling or empty-
 * space skipping.  Images equal those of the flat table. */
#define VOL_LAYOUT_SPARSE_PT 2u

/* Brick-and-level layout that vol_create() would use (pure host computation). */
typedef struct {
    int64_t dims[3];
    int32_t dtype, brick, levels;
    int32_t bytes_per_voxel;
    int32_t layout;        /* 0 quad, 1 compact */
    int32_t entry_voxels;  /* voxels stored per addressable entry: 4 (quad) or 1 */
    int64_t level_dims[VOL_MAX_LEVELS][3];
    int64_t level_bricks[VOL_MAX_LEVELS][3];  /* ceil(D_l / B) per axis */
    int64_t level_pt_offset[VOL_MAX_LEVELS];  /* first page-table entry of each level (sparse: of
                                                 its top grid) */
    int64_t total_bricks;                     /* bricks over all levels (flat: page-table entries) */
    int64_t slot_bytes;   /* one atlas slot: (B+1)^3 voxels, padded to 256 bytes */
    int64_t nslots;       /* atlas capacity in bricks */
    int64_t atlas_bytes;
    int64_t sparse_pt;      /* 1: VOL_LAYOUT_SPARSE_PT */
    int64_t pt_top_entries; /* sparse: entries of the levels' top grids */
} vol_layout;

/* Per-render counters (vol_get_stats). */
typedef struct {
    int64_t passes;          /* kernel passes of the last render (1 when nothing missed) */
    int64_t rays;            /* rays of the last render */
    int64_t suspended;       /* rays suspended at a missing brick, summed over passes */
    int64_t requests;        /* distinct brick requests, summed over passes */
    int64_t request_overflow;/* requests dropped because the table's probe bound was hit */
    int64_t bricks_loaded;   /* bricks the provider filled during the last render */
    int64_t bytes_loaded;    /* host-to-device brick bytes during the last render */
    int64_t evicted;         /* slots evicted during the last render */
    int64_t resident;        /* resident bricks after the last render */
    int64_t frame;           /* frame counter (one per vol_render) */
    int64_t device_error;    /* device-side check failures (0 expected) */
    int64_t touched;         /* distinct bricks the last render sampled (usage stamps) */
    int64_t load_wait_us;    /* host time the last render spent waiting for the provider (us) */
    int64_t launches;        /* kernels the library launched since the last render began */
    int64_t preview_samples; /* preview: samples taken on a coarser level or left out */
    int64_t allocations;     /* device and pinned-host allocations the volume has made since
                                vol_create (cumulative; never reset) */
    int64_t skipped_samples; /* VOL_RENDER_SKIP_EMPTY: samples jumped over (not composited) */
} vol_stats;

/* Provider of bricks that are not resident (procedural or out-of-core source).
 * Fills dst (host memory owned by the library, (B+1)^3 voxels of type
 * src_dtype as declared by vol_set_provider) with the voxels of brick
 * (bx, by, bz) of `level` INCLUDING the one-voxel apron on its +x/+y/+z sides:
 * voxel (i, j, k) of dst, i, j, k in [0, B], is the level voxel
 * (min(bx*B + i, D_l - 1), min(by*B + j, D_l - 1), min(bz*B + k, D_l - 1)).
 * Returns 0 on success. Called from the host thread that called vol_render(). */
typedef int (*vol_provider_fn)(void *user, int level, const int32_t brick[3], void *dst);

/* Batch form of the provider: fills n bricks in one call (so the source can work on them in
 * parallel).  reqs: host int32 [n][4] = level, bx, by, bz; dst: host memory owned by the
 * library (pinned), n consecutive (B+1)^3 regions of src_dtype in request order, each with
 * the voxel contract of vol_provider_fn.  Returns 0 on success. */
typedef int (*vol_provider_batch_fn)(void *user, int n, const int32_t *reqs, void *dst);

/* Debug record of one sample's decisions (vol_trace). */
typedef struct {
    int32_t k;          /* sample index */
    uint32_t t_bits;    /* binary32 bits of t_k */
    int32_t level;      /* LOD level */
    int32_t i0[3];      /* clamped lower-corner voxel on the level grid */
    int32_t local[3];   /* position inside the brick: i0 mod B */
    int32_t pad;
    int64_t brick_id;   /* bx + nbx * (by + nby * bz) on the level */
    uint32_t slot;      /* atlas slot from the page table (0xFFFFFFFF = not resident) */
    uint32_t pad2;
} vol_trace_rec;

/* ---- layout and lifetime ------------------------------------------------ */

/* Computes the layout for dims / dtype / brick (power of two, 4..128) /
 * levels (1..16) / cache_bytes (0 = room for every brick of every level) /
 * flags (VOL_LAYOUT_COMPACT, VOL_LAYOUT_SPARSE_PT or 0): the bricking of
 * Sec. III-A (chunk position h = floor(g / B) per axis), the level dims of
 * Sec. III-D and the page-table extents of Sec. III-E.  Pure host code; needs
 * no GPU.  Errors: VOL_ERR_INVALID_ARG (bad sizes, type or flags),
 * VOL_ERR_UNSUPPORTED (more bricks than the chosen page table can index). */
int vol_plan(const int64_t dims[3], int dtype, int brick, int levels, uint64_t cache_bytes,
             uint32_t flags, vol_layout *out);

/* Creates a volume on the current CUDA device (Sec. III-C: the GPU-side brick
 * store, here an atlas of equal slots; Sec. III-E: one page table per LOD
 * level).  Allocates the atlas (the cache of brick slots), the page tables
 * (all entries non-resident) and the slot usage stamps.  Arguments as for
 * vol_plan(); `stream` is a cudaStream_t or NULL.  *out receives the handle,
 * which the caller releases with vol_destroy().  Errors: those of vol_plan(),
 * VOL_ERR_OOM, VOL_ERR_CUDA (message from vol_last_error(NULL)). */
int vol_create(const int64_t dims[3], int dtype, int brick, int levels, uint64_t cache_bytes,
               uint32_t flags, void *stream, vol_t *out);

/* Frees everything the volume allocated, after waiting for its stream.  NULL
 * is ignored.  (Library plumbing; the paper has no counterpart.) */
void vol_destroy(vol_t v);

/* Message of the last failure on v (or of the last vol_create failure when
 * v is NULL).  Valid until the next call on v.  (Library plumbing; the paper
 * has no counterpart.) */
const char *vol_last_error(vol_t v);

/* Sets the CUDA stream (cudaStream_t or NULL) that orders the volume's later
 * device work.  (Library plumbing; the paper has no counterpart.) */
int vol_set_stream(vol_t v, void *stream);

/* Copies the volume's layout (as vol_plan() computed it) to *out.  (Library
 * plumbing; the paper has no counterpart.) */
int vol_get_layout(vol_t v, vol_layout *out);

/* Copies the counters of the last render to *out; `touched` is read from the
 * per-slot usage stamps (Sec. III-C/III-E use tracking).  Synchronises the
 * stream. */
int vol_get_stats(vol_t v, vol_stats *out);

/* ---- bricks -------------------------------------------------------------- */

/* Sec. III-A bricking and Sec. III-E page-table insertion of a whole level:
 * makes every brick of `level` resident from a dense level array `src`
 * (D_l voxels per axis, x fastest) of type src_dtype, in host memory
 * (src_on_device = 0) or device memory (1).  Each brick is written into its
 * atlas slot with its +side apron (edge voxels replicated at the volume
 * boundary).  Conversions: equal types are copied; u16 -> f16 stores the
 * binary16 of the binary32 quotient u / 65535; u8 -> f32 and u16 -> f32
 * store u / 255 and u / 65535 in binary32; others are VOL_ERR_UNSUPPORTED.
 * Host sources are copied synchronously. */
int vol_upload_level(vol_t v, int level, const void *src, int src_dtype, int src_on_device);

/* Answers a brick request (Sec. III-H) by hand: makes brick (bx, by, bz) of
 * `level` resident from (B+1)^3 voxels (apron included, layout as for
 * vol_provider_fn) of type src_dtype in host (src_on_device = 0, copied
 * before the call returns) or device memory (1, read on the stream) and
 * publishes it in the level's page table (Sec. III-E).  Evicts the least
 * recently used brick when the atlas is full (Sec. III-C).  Errors:
 * VOL_ERR_INVALID_ARG (level or brick out of range), VOL_ERR_UNSUPPORTED
 * (conversion), VOL_ERR_CACHE_FULL, VOL_ERR_CUDA. */
int vol_upload_brick(vol_t v, int level, const int32_t brick[3], const void *src, int src_dtype,
                     int src_on_device);

/* Builds levels from_level+1 .. L-1 from resident level from_level by the
 * 2x2x2 box filter of Sec. III-D: coarse voxel i averages fine voxels 2i and
 * 2i+1 per axis (the last fine voxel replaces an index past the edge);
 * integer types: (sum + 4) >> 3; float types: binary32 sum in (dz, dy, dx)
 * order times 0.125 (binary16 rounded to nearest even).  Every brick of each
 * source level must be resident; all bricks of the built levels become
 * resident.  VOL_ERR_CACHE_FULL when the atlas cannot hold them. */
int vol_build_lod(vol_t v, int from_level);

/* Copies the (B+1)^3 stored voxels of a resident brick (apron included, x
 * fastest, whatever the slot layout) to host memory dst; synchronous.
 * VOL_ERR_INVALID_ARG when not resident.  (A debugging aid; the paper has no
 * counterpart.) */
int vol_download_brick(vol_t v, int level, const int32_t brick[3], void *dst);

/* Drops every brick: page tables back to non-resident (Sec. III-E), every
 * slot free (Sec. III-C).  Enqueued on the stream. */
int vol_evict_all(vol_t v);

/* Installs (or with fn = NULL removes) the provider used by vol_render() to
 * load missing bricks: the source that answers the brick requests of
 * Sec. III-H, e.g. chunks generated on the fly as in Sec. V-C.  src_dtype is
 * the type the provider writes; `user` is passed back to it unchanged and is
 * owned by the caller. */
int vol_set_provider(vol_t v, vol_provider_fn fn, void *user, int src_dtype);

/* Installs (or with fn = NULL removes) a batch provider (the source of Sec. III-H's brick
 * requests, called for many bricks at once; Sec. V-C's on-the-fly chunk generation); it takes
 * precedence over the per-brick provider.  Bricks are requested in batches of up to 64 MiB of
 * source voxels.  `user` is owned by the caller and must outlive the volume's use of it. */
int vol_set_provider_batch(vol_t v, vol_provider_batch_fn fn, void *user, int src_dtype);

/* ---- rendering ----------------------------------------------------------- */

/* Direct volume rendering (Sec. IV-A; ray entry/exit and camera of Fig. 1;
 * footprint LOD of Sec. V-C; brick requests of Sec. III-H; tiles as tasks of
 * Sec. III-H).  Renders nviews views (cams: host array) in one persistent
 * launch that takes ray tiles of all views from one work counter.  tf_dev: device
 * float [256][4] RGBA transfer function (entry j at value j / 255, linearly
 * interpolated).  rgba_dev: output float [pixels][4], the views' images
 * packed in order, in memory of the volume's GPU or in page-locked host
 * memory (cudaHostAlloc / cudaHostRegister; the kernel then writes the image
 * through its device mapping across the host link, so the result needs no
 * copy and is complete when the volume's stream is); any other pointer gives
 * VOL_ERR_INVALID_ARG before any launch.  nsamples_dev: optional int32 per
 * pixel, the number of samples composited (NULL to skip), in the same kinds
 * of memory.
 * Sample k of a ray is at t_k = t0 + k * step while t_k < t1 (entry/exit of
 * the box); C += T a rgb, T *= 1 - a; the ray stops after the sample where
 * 1 - T >= et_threshold; output rgb = C + T bg_rgb, a = (1 - T) + T bg_a.
 * When every brick is resident the call only enqueues work.  Otherwise it
 * synchronises: rays that reach a missing brick are suspended (position and
 * partial colour kept), the bricks are requested through a deduplicating
 * hash table, and -- if a provider is set -- loaded and the suspended rays
 * resumed, up to max_passes passes; without a provider, or when passes run
 * out, it returns VOL_ERR_INCOMPLETE and the requests can be read with
 * vol_poll_requests().  The finished image does not depend on how many
 * passes it took. */
int vol_render(vol_t v, const vol_camera *cams, int nviews, const float *tf_dev,
               const vol_params *params, float *rgba_dev, int32_t *nsamples_dev);

/* Resumes the rays that the last vol_render() left suspended, after the
 * caller uploaded the requested bricks (vol_upload_brick): the kernel run
 * again after the requests are answered, Sec. III-H.  Synchronises.
 * VOL_OK when every ray finished, else VOL_ERR_INCOMPLETE;
 * VOL_ERR_NO_FORWARD_STATE without a render. */
int vol_render_resume(vol_t v);

/* Reads the brick-request table of Sec. III-H: copies up to cap outstanding
 * brick requests of the last pass as [level, bx, by, bz] int32 quadruples to
 * host memory `out` (caller-owned, cap * 4 int32); *n receives their total
 * count (which may exceed cap).  Synchronises.  VOL_ERR_INVALID_ARG for a
 * NULL n, or a NULL out with cap > 0. */
int vol_poll_requests(vol_t v, int32_t *out, int cap, int *n);

/* Adjoint of the last vol_render() made with VOL_RENDER_GRAD (every brick of
 * the levels it sampled still resident, no suspended rays).  Not in the paper:
 * the reverse of Sec. IV-A's front-to-back compositing.  drgba_dev: dL/dRGBA in
 * the layout of rgba_dev.  Accumulates (+=) dL/dtf into dtf_dev (device float
 * [256][4]) and dL/dvoxel into dvoxel_dev (device float, dense level 0, x
 * fastest; gradient with respect to the normalised voxel value).  Either
 * output may be NULL.  Transmittance is recomputed forward from checkpoints
 * stored every 32 samples, never by dividing by (1 - a).  With footprint LOD
 * (lod_mode 1) a sample on level l reads level-l voxels, each the 2x2x2 box
 * filter of level l-1 (Sec. III-D): their gradients are carried down to level
 * 0 through the filter's adjoint, 1/8 to each child (a child index past an
 * odd edge counts as the last voxel, as in the filter; integer storage is
 * differentiated as the mean).  Errors: VOL_ERR_NO_FORWARD_STATE (no gradient
 * render, an incomplete one, or a level evicted since), VOL_ERR_INVALID_ARG
 * (NULL drgba_dev), VOL_ERR_CUDA. */
int vol_render_backward(vol_t v, const float *drgba_dev, float *dtf_dev, float *dvoxel_dev);

/* Debug: the decision-layer record (sample depth, Sec. V-C footprint level,
 * Sec. III-A voxel, brick and local position, Sec. III-E slot) of up to
 * max_samples samples of each of npix pixels (pixels_host: int32 [npix][2] =
 * px, py of view `cam`), without early termination.  out_host: [npix][max_samples] records; counts_host:
 * int32 [npix] total samples per ray.  Synchronises. */
int vol_trace(vol_t v, const vol_camera *cam, const vol_params *params, const int32_t *pixels_host,
              int npix, int max_samples, vol_trace_rec *out_host, int32_t *counts_host);

/* ---- rendering without any allocation ------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory once set-up is over: a host application that
 * reserves its whole device-memory budget up front and refuses later
 * allocations, or a render loop that must never stall inside the allocator.
 * vol_render() may allocate on its first calls (its view table, and, for
 * partly resident volumes or gradient mode, request tables, suspended-ray
 * buffers and checkpoints); this variant never does.
 *
 * It renders like vol_render() (same kernel, same image) from a volume whose
 * bricks are all resident for the levels the parameters use.  Its only scratch
 * (the work counter and the view table) lives in one static device array of
 * VOL_NOALLOC_SCRATCH_BYTES (8 KiB) inside the library, which every GPU that
 * loads the library keeps until the process exits; hence at most
 * VOL_NOALLOC_MAX_VIEWS views per call.  The caller passes inputs and outputs
 * exactly as for vol_render().
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current.
 *   - All calls share the array, and each call overwrites it: calls that
 *     overlap on the GPU (different streams, or different volumes on streams
 *     that are not ordered) race.  Calls on one stream are ordered and safe.
 *   - It neither queues brick requests nor keeps state for
 *     vol_render_backward(), and it does not update the LRU usage stamps.
 * Errors: VOL_ERR_INVALID_ARG (null pointers, an output the GPU cannot address, nviews outside
 * 1..VOL_NOALLOC_MAX_VIEWS, bad image size or tile), VOL_ERR_UNSUPPORTED
 * (VOL_RENDER_GRAD set, a needed level not fully resident, or a sparse page
 * table with a projection or level-scaled sampling), VOL_ERR_CUDA.
 * vol_stats then describes this call (launches = 1), and
 * vol_stats.allocations stays unchanged. */
#define VOL_NOALLOC_SCRATCH_BYTES 8192
#define VOL_NOALLOC_MAX_VIEWS 64
int vol_render_noalloc(vol_t v, const vol_camera *cams, int nviews, const float *tf_dev,
                       const vol_params *params, float *rgba_dev, int32_t *nsamples_dev);

#ifdef __cplusplus
}
#endif
#endif /* VOLRC_VOL_H */
