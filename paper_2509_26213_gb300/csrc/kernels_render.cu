// kernels_render.cu -- variants of the forward kernel for emission/absorption compositing
// (with and without gradient checkpoints), the adjoint, the longest-ray-first tile order and
// the decision trace.  The forward kernel template and its building blocks are in
// render_common.cuh.
#include "render_common.cuh"

namespace volrc {
namespace {

// ------------------------------------------------------------------ adjoint

// dL/dtf accumulates in shared memory channel-major (s_dtf[c * 256 + i]), so that lanes
// flushing different entries of one channel fall into different banks.  The table is kept in
// DtfTable::kCopies copies, lane l adding to copy l % kCopies, each copy shifted by 32 / kCopies
// banks: neighbouring rays often flush the same entry at once, and additions to one address in
// one instruction are serialised.  The copies are summed at the end.
__device__ __forceinline__ void flush_dtf(float* s_dtf, int idx, float acc[8]) {
    if (idx >= 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (acc[c] != 0.0f) atomicAdd(&s_dtf[c * 256 + idx], acc[c]);
            if (acc[4 + c] != 0.0f) atomicAdd(&s_dtf[c * 256 + idx + 1], acc[4 + c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
}

// Adds the corner accumulators of trilinear cell `cell` (linear index of its lower corner;
// cacc[cx + 2 cy + 4 cz]; mask: which +1 corners exist) to dvox, row by row (x-neighbour
// pairs), skipping rows that do not exist or hold only zeros.  (16-byte vector atomics for the
// pairs measured 2% slower than these scalar ones on the 16 x 512^2 workload.)
__device__ __forceinline__ void flush_vox(float* dvox, long long cell, int mask, int Dx, int Dy, float cacc[8]) {
    if (cell >= 0) {
        const long long sy = Dx, sz = (long long)Dx * Dy;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int cy = r & 1, cz = r >> 1;
            const bool row_ok = (!cy || (mask & 2)) && (!cz || (mask & 4));
            const float v0 = cacc[2 * r], v1 = (mask & 1) ? cacc[2 * r + 1] : 0.0f;
            if (!row_ok || (v0 == 0.0f && v1 == 0.0f)) continue;
            const long long L = cell + cy * sy + cz * sz;
            if (v0 != 0.0f) atomicAdd(dvox + L, v0);
            if (v1 != 0.0f) atomicAdd(dvox + L + 1, v1);
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) cacc[c] = 0.0f;
}

// Adds the 4 accumulators of one entry (acc[0..3], one per channel) to dL/dtf.
__device__ __forceinline__ void flush_dtf4(float* s_dtf, int idx, const float* acc) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (acc[c] != 0.0f) atomicAdd(&s_dtf[c * 256 + idx], acc[c]);
}

// Copies of the dL/dtf table: with the value tape the segment's values are not kept in shared
// memory, which leaves room for 4 copies at the same occupancy.
#ifndef VOLRC_BWD_COPIES
#define VOLRC_BWD_COPIES 4
#endif
template <bool TAPE>
struct DtfTable {
    static constexpr int kCopies = TAPE ? VOLRC_BWD_COPIES : 1;
    static constexpr int kStride = 1024 + (kCopies > 1 ? 32 / kCopies : 0);  // words between copies
};

// Samples per lane whose page-table lookups and gathers the adjoint's forward recompute issues
// together.
#ifndef VOLRC_BWD_BATCH
#define VOLRC_BWD_BATCH 4
#endif
constexpr int kBwdBatch = VOLRC_BWD_BATCH;
// Adjoint CTA size and the resident CTAs per SM its register allocation must allow (shared
// memory per CTA: 4 KiB + 4 KiB per dL/dtf copy + 256 B per thread).
#ifndef VOLRC_BWD_THREADS
#define VOLRC_BWD_THREADS 192
#endif
#ifndef VOLRC_BWD_MINB
#define VOLRC_BWD_MINB 4
#endif
constexpr int kBwdThreads = VOLRC_BWD_THREADS;
constexpr int kBwdMinBlocks = VOLRC_BWD_MINB;

// Adjoint, warp-synchronous by checkpoint segment: a warp takes 32 rays (a ray tile, or a
// 32-pixel part of it) and, round by round, processes segment s of every one of them that has
// it (samples 32 s .. 32 s + 31, the last one partial), s descending from the longest ray's last
// segment: first forward -- transmittance from the segment's checkpoint and the sample values
// into shared memory, kBwdBatch samples at a time -- then in reverse, accumulating dL/dtf and
// dL/dvoxel.  Neighbouring rays then sample neighbouring depths in each round, as in the forward
// march, which keeps the gathers and the dL/dvoxel reductions of a round together in the cache.
// (With checkpoints before every sample -- the store-all debug mode -- a segment is one sample
// and its transmittance is read, not recomputed.)
// LOD: samples on footprint levels; the gradient of a level-l voxel goes to P.dlev[l], which
// the host then carries down to level 0 through the box filter's adjoint.
// TAPE: the segment's sample values are read from the forward's value tape instead of being
// interpolated again from the bricks (the transmittance is recomputed from the checkpoint either way).
template <int DT, bool LOD, bool TAPE>
__global__ void __launch_bounds__(kBwdThreads, kBwdMinBlocks) k_backward(const __grid_constant__ BackwardDev P) {
    __shared__ float4 s_tf[256];
    constexpr int kDtfCopies = DtfTable<TAPE>::kCopies, kDtfStride = DtfTable<TAPE>::kStride;
    __shared__ float s_dtf_all[kDtfCopies * kDtfStride];
    __shared__ float s_T[kCkptEvery][kBwdThreads];
    __shared__ float s_V[TAPE ? 1 : kCkptEvery][kBwdThreads];  // (with the tape: read from it again)
    __shared__ LevelDev s_lv[LOD ? kMaxLevels : 1];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tf[i] = P.tf[i];
    for (int i = threadIdx.x; i < kDtfCopies * kDtfStride; i += blockDim.x) s_dtf_all[i] = 0.0f;
    float* s_dtf = s_dtf_all + (threadIdx.x & 31) % kDtfCopies * kDtfStride;  // this lane's copy
    if (LOD && threadIdx.x < P.vol.nlevels) s_lv[threadIdx.x] = P.vol.lv[threadIdx.x];
    __syncthreads();

    using VT = typename Voxel<DT>::T;
    const VT* __restrict__ atlas = (const VT*)P.vol.atlas;
    const unsigned lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const int bshift = P.vol.bshift, bmask = P.vol.bmask, B1 = P.vol.B1;
    const bool quad = P.vol.quad != 0;
    const int row = quad ? B1 - 1 : B1;
    const unsigned long long slot_stride = quad ? P.vol.slot_entries : P.vol.slot_elems;
    LvReg L0 = load_lv(P.vol.lv[0]);  // LOD: the level of the last resolved sample
    // voxels along x and y of level l (the shared level table when LOD)
    auto dim_x = [&](int l) { return LOD ? s_lv[l].D[0] : P.vol.lv[0].D[0]; };
    auto dim_y = [&](int l) { return LOD ? s_lv[l].D[1] : P.vol.lv[0].D[1]; };
    int cur_l = 0;
    const int nlev = P.vol.nlevels;
    const float step = P.step;
    // per-lane accumulators: dL/dtf for entries acc_i, acc_i + 1; dL/dvoxel for the 8 corners
    // of cell cell_cur on level cell_lvl (cell_mask: which +1 corners exist)
    int acc_i = -1;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    long long cell_cur = -1;
    int cell_mask = 0, cell_lvl = 0;
    float cacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    // lane state: the lane's ray, its sample count n and segment count nseg
    bool has = false;
    long long ray = 0;
    float o0 = 0, o1 = 0, o2 = 0, d0 = 0, d1 = 0, d2 = 0, t0 = 0, lodscale = 0;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    float R0 = 0, R1 = 0, R2 = 0, R3 = 0;
    int n = 0, nseg = 0;
    // warp-uniform: the segment index every lane processes in this round, descending; each
    // lane's rays sample the same depths as its neighbours' (adjacent pixels), so the gathers
    // and the dL/dvoxel reductions of a round stay close together in the volume
    int s = -1;
    const int tile_px = P.tile_w * P.tile_h;
    const int chunks = (tile_px + 31) >> 5;  // work items per tile: 32 rays each

    for (;;) {
        if (s < 0) {
            // ---- the next 32 rays: one tile, or a 32-pixel part of a larger one
            int item = 0;
            if (lane == 0) item = (int)atomicAdd(&P.counters[kWork], 1u);
            item = __shfl_sync(kFull, item, 0);
            if (item >= P.nwork) break;
            const int ti = item / chunks, part = item - ti * chunks;
            const int tile = P.tile_order ? P.tile_order[ti] : ti;
            const int v = find_view_tile(P.views, P.nviews, tile);
            const ViewDev& V = P.views[v];
            const int tl = tile - V.tile_off;
            const int idx = part * 32 + (int)lane;
            const int px = (tl % V.tiles_x) * P.tile_w + idx % P.tile_w;
            const int py = (tl / V.tiles_x) * P.tile_h + idx / P.tile_w;
            has = false;
            nseg = 0;
            if (idx < tile_px && px < V.w && py < V.h) {
                ray = V.ray_off + (long long)py * V.w + px;
                n = P.ray_n[ray];
                if (n > 0) {
                    Ray R;
                    make_ray(V, P.vol.D0f, px, py, R);
                    o0 = R.o[0]; o1 = R.o[1]; o2 = R.o[2];
                    d0 = R.d[0]; d1 = R.d[1]; d2 = R.d[2];
                    t0 = R.t0;
                    lodscale = V.lodscale;
                    g = P.drgba[ray];
                    R0 = P.bg.x; R1 = P.bg.y; R2 = P.bg.z; R3 = P.bg.w;
                    nseg = ((n - 1) >> P.ckpt_shift) + 1;
                    has = true;
                }
            }
            s = __reduce_max_sync(kFull, nseg) - 1;
            if (s < 0) continue;
        }

        // ---- one round: segment s (2^ckpt_shift <= kCkptEvery samples) of every lane's ray that has it
        const bool seg = has && s < nseg;
        const int k0 = s << P.ckpt_shift;
        const int len = seg ? min(1 << P.ckpt_shift, n - k0) : 0;
        float T = (seg && s > 0) ? P.ckpt[(long long)(s - 1) * P.nrays + ray] : 1.0f;
        const int maxlen = __reduce_max_sync(kFull, len);
        // the lane's segment on the tape: 32 values in 128 contiguous bytes
        const float* tp = TAPE ? P.tape + ((long long)s * P.nrays + (seg ? ray : 0)) * kCkptEvery : nullptr;
        if (TAPE) {
            // forward from the tape, 4 values per load
            for (int jb = 0; jb < maxlen; jb += 4) {
                const float4 v4 = jb < len ? __ldg(reinterpret_cast<const float4*>(tp + jb)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jb + u < len) {
                        const float x = tf_coord<DT>(vv[u]);
                        const int i = min((int)x, 254);
                        const float wt = x - (float)i;
                        const float al = fmaf(wt, s_tf[i + 1].w - s_tf[i].w, s_tf[i].w);
                        s_T[jb + u][tid] = T;
                        T = T * (1.0f - al);
                    }
                }
            }
        }
        // forward: decisions, then the page-table lookups, then the gathers of kBwdBatch samples
        for (int jb = 0; !TAPE && jb < maxlen; jb += kBwdBatch) {
            uint32_t pti[kBwdBatch], loc[kBwdBatch];
            float wv[kBwdBatch][3];
            const float kf = (float)(k0 + jb);  // + u stays exact: indices are below 2^24
#pragma unroll
            for (int u = 0; u < kBwdBatch; ++u) {
                const float t = __fadd_rn(t0, __fmul_rn(__fadd_rn(kf, (float)u), step));
                const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)),
                                    __fadd_rn(o2, __fmul_rn(t, d2))};
                if (LOD) {
                    const int l = lod_level(t, lodscale, P.lod_bias, nlev);
                    if (l != cur_l) {
                        cur_l = l;
                        L0 = load_lv(s_lv[l]);
                    }
                }
                Resolved Q;
                resolve_reg(L0, bshift, bmask, row, p, Q);
                pti[u] = Q.pti;
                loc[u] = Q.local;
                wv[u][0] = Q.w[0];
                wv[u][1] = Q.w[1];
                wv[u][2] = Q.w[2];
            }
            uint32_t slot[kBwdBatch];
#pragma unroll
            for (int u = 0; u < kBwdBatch; ++u) slot[u] = __ldg(P.vol.pt + (jb + u < len ? pti[u] : 0u));
            float val[kBwdBatch];
#pragma unroll
            for (int u = 0; u < kBwdBatch; ++u) {
                const bool use = jb + u < len && slot[u] != kInvalidSlot;
                const unsigned long long base = use ? (unsigned long long)slot[u] * slot_stride + loc[u] : 0ull;
                val[u] = quad ? trilinear_quad<DT>(P.vol.atlas, base, B1 - 1, wv[u])
                              : trilinear<DT>(atlas, base, B1, wv[u]);
            }
#pragma unroll
            for (int u = 0; u < kBwdBatch; ++u) {
                if (jb + u < len) {
                    if (slot[u] == kInvalidSlot) atomicAdd(&P.counters[kDevError], 1u);
                    const float x = tf_coord<DT>(val[u]);
                    const int i = min((int)x, 254);
                    const float wt = x - (float)i;
                    const float al = fmaf(wt, s_tf[i + 1].w - s_tf[i].w, s_tf[i].w);
                    s_T[jb + u][tid] = T;
                    if (!TAPE) s_V[jb + u][tid] = val[u];
                    T = T * (1.0f - al);
                }
            }
        }
        float kf = (float)(k0 + maxlen - 1);  // (float)(k0 + j), stepped down exactly
        for (int j = maxlen - 1; j >= 0; --j, kf = __fsub_rn(kf, 1.0f)) {
            if (j < len) {
                Resolved Q;  // the sample's voxel and weights: only dL/dvoxel needs them
                if (P.dvox) {
                    const float t = __fadd_rn(t0, __fmul_rn(kf, step));
                    const float p[3] = {__fadd_rn(o0, __fmul_rn(t, d0)), __fadd_rn(o1, __fmul_rn(t, d1)),
                                        __fadd_rn(o2, __fmul_rn(t, d2))};
                    if (LOD) {
                        const int l = lod_level(t, lodscale, P.lod_bias, nlev);
                        if (l != cur_l) {
                            cur_l = l;
                            L0 = load_lv(s_lv[l]);
                        }
                    }
                    resolve_reg(L0, bshift, bmask, row, p, Q);
                }
                const float val = TAPE ? __ldg(tp + j) : s_V[j][tid];
                const float Tk = s_T[j][tid];
                const float x = tf_coord<DT>(val);
                const int i = min((int)x, 254);
                const float wt = x - (float)i;
                const float4 a = s_tf[i], b = s_tf[i + 1];
                const float cr = fmaf(wt, b.x - a.x, a.x), cg = fmaf(wt, b.y - a.y, a.y);
                const float cb = fmaf(wt, b.z - a.z, a.z), al = fmaf(wt, b.w - a.w, a.w);
                const float dal = Tk * (g.x * (cr - R0) + g.y * (cg - R1) + g.z * (cb - R2) + g.w * (1.0f - R3));
                const float Ta = Tk * al;
                const float dr = g.x * Ta, dg = g.y * Ta, db = g.z * Ta;
                if (P.dtf) {
                    // register accumulation while the TF index stays the same
                    if (i != acc_i) {
                        // to a neighbouring index the entry both lookups share stays in registers:
                        // only the one left behind is added to the table
                        if (acc_i >= 0 && i == acc_i + 1) {
                            flush_dtf4(s_dtf, acc_i, acc);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc[c] = acc[4 + c];
                                acc[4 + c] = 0.0f;
                            }
                        } else if (acc_i >= 0 && i == acc_i - 1) {
                            flush_dtf4(s_dtf, acc_i + 1, acc + 4);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc[4 + c] = acc[c];
                                acc[c] = 0.0f;
                            }
                        } else {
                            flush_dtf(s_dtf, acc_i, acc);
                        }
                        acc_i = i;
                    }
                    const float w0 = 1.0f - wt;
                    acc[0] = fmaf(w0, dr, acc[0]);
                    acc[1] = fmaf(w0, dg, acc[1]);
                    acc[2] = fmaf(w0, db, acc[2]);
                    acc[3] = fmaf(w0, dal, acc[3]);
                    acc[4] = fmaf(wt, dr, acc[4]);
                    acc[5] = fmaf(wt, dg, acc[5]);
                    acc[6] = fmaf(wt, db, acc[6]);
                    acc[7] = fmaf(wt, dal, acc[7]);
                }
                if (P.dvox && tf_inside<DT>(val)) {
                    const float dv = 255.0f * (dr * (b.x - a.x) + dg * (b.y - a.y) + db * (b.z - a.z) + dal * (b.w - a.w));
                    if (dv != 0.0f) {
                        // register accumulation while the trilinear cell (and level) stays the same
                        const int lq = LOD ? cur_l : 0;
                        const int Dx = (int)L0.Dm[0] + 1, Dy = (int)L0.Dm[1] + 1;
                        const long long cell = (long long)Q.i0[0] + (long long)Dx * ((long long)Q.i0[1] + (long long)Dy * Q.i0[2]);
                        if (cell != cell_cur || lq != cell_lvl) {
                            flush_vox(P.dlev[cell_lvl], cell_cur, cell_mask, dim_x(cell_lvl), dim_y(cell_lvl), cacc);
                            cell_cur = cell;
                            cell_lvl = lq;
                            cell_mask = ((float)Q.i0[0] < L0.Dm[0] ? 1 : 0) | ((float)Q.i0[1] < L0.Dm[1] ? 2 : 0) |
                                        ((float)Q.i0[2] < L0.Dm[2] ? 4 : 0);
                        }
                        const float wx = Q.w[0], wy = Q.w[1], wz = Q.w[2];
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
                            const float wgt = (cx ? wx : 1.0f - wx) * (cy ? wy : 1.0f - wy) * (cz ? wz : 1.0f - wz);
                            cacc[c] = fmaf(wgt, dv, cacc[c]);
                        }
                    }
                }
                R0 = fmaf(al, cr - R0, R0);
                R1 = fmaf(al, cg - R1, R1);
                R2 = fmaf(al, cb - R2, R2);
                R3 = fmaf(al, 1.0f - R3, R3);
            }
        }
        --s;
    }
    if (P.dtf) flush_dtf(s_dtf, acc_i, acc);
    if (P.dvox) flush_vox(P.dlev[cell_lvl], cell_cur, cell_mask, dim_x(cell_lvl), dim_y(cell_lvl), cacc);
    __syncthreads();
    if (P.dtf)
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
            float v = 0.0f;
#pragma unroll
            for (int r = 0; r < kDtfCopies; ++r) v += s_dtf_all[r * kDtfStride + (i & 3) * 256 + (i >> 2)];
            if (v != 0.0f) atomicAdd(&P.dtf[i], v);
        }
}

// ------------------------------------------------------------------ scheduling

// Work order for the next frame: tiles bucketed by floor(log2(cost + 1)), buckets in descending
// order, where a tile's cost is the sample count of its longest ray.  The longest rays start
// first, so none of them begins near the end of the launch and runs on while other SMs idle
// (ordering by the tile's total samples instead left a tail: c2 0.91 -> 0.81 ms with this key).
constexpr int kOrderThreads = 256;

__device__ __forceinline__ int cost_bucket(int c) { return 31 - __clz(c + 1); }

// buckets[0..31]: tiles per bucket; one thread per tile, one global atomic per bucket per block
__global__ void __launch_bounds__(kOrderThreads) k_order_count(const int* cost, int ntiles, int* buckets) {
    __shared__ int s_count[32];
    if (threadIdx.x < 32) s_count[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ntiles) atomicAdd(&s_count[cost_bucket(cost[i])], 1);
    __syncthreads();
    if (threadIdx.x < 32 && s_count[threadIdx.x]) atomicAdd(&buckets[threadIdx.x], s_count[threadIdx.x]);
}

// order[] = tiles grouped by bucket, highest bucket first; each block reserves its places in
// every bucket with one atomic on the bucket's fill cursor (buckets[32 + b]).  Zeroes cost[].
__global__ void __launch_bounds__(kOrderThreads) k_order_scatter(int* cost, int* order, int ntiles, int* buckets) {
    __shared__ int s_count[32], s_base[32];
    if (threadIdx.x < 32) s_count[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = i < ntiles ? cost_bucket(cost[i]) : 0;
    const int rank = i < ntiles ? atomicAdd(&s_count[b], 1) : 0;
    __syncthreads();
    if (threadIdx.x < 32) {
        int base = 0;
        for (int q = 31; q > (int)threadIdx.x; --q) base += buckets[q];
        s_base[threadIdx.x] = s_count[threadIdx.x] ? base + atomicAdd(&buckets[32 + threadIdx.x], s_count[threadIdx.x]) : 0;
    }
    __syncthreads();
    if (i < ntiles) {
        order[s_base[b] + rank] = i;
        cost[i] = 0;
    }
}

// ------------------------------------------------------------------ trace

__global__ void k_trace(const __grid_constant__ TraceDev P) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P.npix) return;
    Ray R;
    make_ray(P.view, P.vol.D0f, P.pixels[2 * q], P.pixels[2 * q + 1], R);
    int k = 0;
    if (R.hit) {
        float t = R.t0;
        int l = 0;
        for (;; ++k) {
            t = P.level_step ? (k ? next_t_level_step(t, P.step, l) : R.t0) : __fadd_rn(R.t0, __fmul_rn((float)k, P.step));
            if (!(t < R.t1)) break;
            l = P.lod_mode ? lod_level(t, P.view.lodscale, P.lod_bias, P.vol.nlevels) : 0;
            if (k >= P.max_samples) continue;
            const float p[3] = {__fadd_rn(R.o[0], __fmul_rn(t, R.d[0])), __fadd_rn(R.o[1], __fmul_rn(t, R.d[1])),
                                __fadd_rn(R.o[2], __fmul_rn(t, R.d[2]))};
            const LevelDev& L = P.vol.lv[l];
            Resolved Q;
            resolve(L, P.vol.bshift, P.vol.bmask, P.vol.quad ? P.vol.B1 - 1 : P.vol.B1, p, Q);
            vol_trace_rec rec;
            rec.k = k;
            rec.t_bits = __float_as_uint(t);
            rec.level = l;
            for (int a = 0; a < 3; ++a) {
                rec.i0[a] = Q.i0[a];
                rec.local[a] = Q.i0[a] & P.vol.bmask;
            }
            rec.pad = 0;
            if (P.vol.sparse) {
                const int h0 = Q.i0[0] >> P.vol.bshift, h1 = Q.i0[1] >> P.vol.bshift, h2 = Q.i0[2] >> P.vol.bshift;
                rec.brick_id = (int64_t)h0 + (int64_t)L.nb[0] * ((int64_t)h1 + (int64_t)L.nb[1] * h2);
                uint32_t leaf;
                rec.slot = sparse_walk(P.vol.pt, load_lv(L), h0, h1, h2, leaf);
            } else {
                rec.brick_id = (int64_t)(Q.pti - L.pt_off);
                rec.slot = P.vol.pt[Q.pti];
            }
            rec.pad2 = 0;
            P.out[(long long)q * P.max_samples + k] = rec;
        }
    }
    P.counts[q] = k;
}

template <int DT, int BS, bool Q>
const void* pick_render_b(bool lod, bool grad) {
    if (grad) return lod ? (const void*)k_render<DT, true, kDvrGrad, BS, Q> : (const void*)k_render<DT, false, kDvrGrad, BS, Q>;
    return lod ? (const void*)k_render<DT, true, kDvr, BS, Q> : (const void*)k_render<DT, false, kDvr, BS, Q>;
}

// quad layout: specialised for bricks of 32 and 64; compact layout: any brick size
template <int DT>
const void* pick_render_d(int brick, bool quad, bool lod, bool grad) {
    if (!quad) return pick_render_b<DT, 0, false>(lod, grad);
    if (brick == 32) return pick_render_b<DT, 32, true>(lod, grad);
    if (brick == 64) return pick_render_b<DT, 64, true>(lod, grad);
    return pick_render_b<DT, 0, true>(lod, grad);
}

const void* pick_render(int dtype, int brick, bool quad, bool lod, bool grad) {
    switch (dtype) {
    case VOL_U8: return pick_render_d<VOL_U8>(brick, quad, lod, grad);
    case VOL_U16: return pick_render_d<VOL_U16>(brick, quad, lod, grad);
    case VOL_F16: return pick_render_d<VOL_F16>(brick, quad, lod, grad);
    case VOL_F32: return pick_render_d<VOL_F32>(brick, quad, lod, grad);
    }
    return nullptr;
}

template <bool LOD, bool TAPE>
const void* pick_backward_l(int dtype) {
    switch (dtype) {
    case VOL_U8: return (const void*)k_backward<VOL_U8, LOD, TAPE>;
    case VOL_U16: return (const void*)k_backward<VOL_U16, LOD, TAPE>;
    case VOL_F16: return (const void*)k_backward<VOL_F16, LOD, TAPE>;
    case VOL_F32: return (const void*)k_backward<VOL_F32, LOD, TAPE>;
    }
    return nullptr;
}

const void* pick_backward(int dtype, bool lod, bool tape) {
    if (tape) return lod ? pick_backward_l<true, true>(dtype) : pick_backward_l<false, true>(dtype);
    return lod ? pick_backward_l<true, false>(dtype) : pick_backward_l<false, false>(dtype);
}

}  // namespace

cudaError_t launch_render(int dtype, int mode, const RenderDev& p, int grid, cudaStream_t s) {
    const void* fn = nullptr;
    // empty-space skipping: flat page table, uniform steps (a quad layout with bricks other than
    // 32 or 64 has no such variant and renders without it; the image is the same)
    if (p.skip_empty && !p.vol.sparse && !p.level_step)
        fn = (mode == kMop || mode == kMip) ? pick_render_skip_projection(dtype, p.vol.B1 - 1, p.vol.quad != 0,
                                                                          p.lod_mode != 0, mode)
                                            : pick_render_skip(dtype, p.vol.B1 - 1, p.vol.quad != 0, p.lod_mode != 0,
                                                               mode);
    if (fn) {
    } else if (mode == kMop || mode == kMip)
        fn = pick_render_projection(dtype, p.vol.B1 - 1, p.vol.quad != 0, p.lod_mode != 0, mode);
    else if (p.vol.sparse && mode == kDvr && !p.level_step)
        fn = pick_render_sparse(dtype, p.vol.B1 - 1, p.vol.quad != 0, p.lod_mode != 0);
    else if (p.vol.sparse)
        fn = nullptr;  // the sparse table has only the emission/absorption variant
    else if (p.level_step && mode == kDvr)
        fn = pick_render_level_step(dtype, p.vol.B1 - 1, p.vol.quad != 0, p.lod_mode != 0);
    else if (!p.level_step)
        fn = pick_render(dtype, p.vol.B1 - 1, p.vol.quad != 0, p.lod_mode != 0, mode == kDvrGrad);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kRenderThreads), args, 0, s);
}

cudaError_t launch_backward(int dtype, const BackwardDev& p, int grid, cudaStream_t s) {
    const void* fn = pick_backward(dtype, p.lod_mode != 0, p.tape != nullptr);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBwdThreads), args, 0, s);
}

cudaError_t launch_tile_order(int* cost, int* order, int ntiles, int* buckets, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(buckets, 0, sizeof(int) * 64, s);
    if (e != cudaSuccess) return e;
    const int grid = (ntiles + kOrderThreads - 1) / kOrderThreads;
    k_order_count<<<grid, kOrderThreads, 0, s>>>(cost, ntiles, buckets);
    k_order_scatter<<<grid, kOrderThreads, 0, s>>>(cost, order, ntiles, buckets);
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceDev& p, cudaStream_t s) {
    const int threads = 64;
    k_trace<<<(p.npix + threads - 1) / threads, threads, 0, s>>>(p);
    return cudaGetLastError();
}

int render_blocks_per_sm(int dtype, bool grad) {
    int n = 0;
    const void* fn = pick_render(dtype, 64, true, false, grad);
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kRenderThreads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

int backward_blocks_per_sm(int dtype, bool lod, bool tape) {
    int n = 0;
    const void* fn = pick_backward(dtype, lod, tape);
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBwdThreads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace volrc
