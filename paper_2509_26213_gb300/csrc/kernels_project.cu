// kernels_project.cu -- variants of the forward kernel for maximum-opacity projection (MOP,
// the compositing of the paper's Kidney renderings, Sec. V-A and Table I) and
// maximum-intensity projection (MIP).  Kept apart from kernels_render.cu so that the two
// sets of template instances compile in parallel.
#include "render_common.cuh"

namespace volrc {
namespace {

template <int DT, int BS, bool Q>
const void* pick_b(bool lod, int mode) {
    if (mode == kMop)
        return lod ? (const void*)k_render<DT, true, kMop, BS, Q> : (const void*)k_render<DT, false, kMop, BS, Q>;
    return lod ? (const void*)k_render<DT, true, kMip, BS, Q> : (const void*)k_render<DT, false, kMip, BS, Q>;
}

template <int DT>
const void* pick_d(int brick, bool quad, bool lod, int mode) {
    if (!quad) return pick_b<DT, 0, false>(lod, mode);
    if (brick == 32) return pick_b<DT, 32, true>(lod, mode);
    if (brick == 64) return pick_b<DT, 64, true>(lod, mode);
    return pick_b<DT, 0, true>(lod, mode);
}

}  // namespace

const void* pick_render_projection(int dtype, int brick, bool quad, bool lod, int mode) {
    if (mode != kMop && mode != kMip) return nullptr;
    switch (dtype) {
    case VOL_U8: return pick_d<VOL_U8>(brick, quad, lod, mode);
    case VOL_U16: return pick_d<VOL_U16>(brick, quad, lod, mode);
    case VOL_F16: return pick_d<VOL_F16>(brick, quad, lod, mode);
    case VOL_F32: return pick_d<VOL_F32>(brick, quad, lod, mode);
    }
    return nullptr;
}

}  // namespace volrc
