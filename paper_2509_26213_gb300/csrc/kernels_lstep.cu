// kernels_lstep.cu -- variants of the forward kernel for level-scaled sampling: a sample on
// LOD level l stands for 2^l reference steps (the next sample is dt * 2^l further and its
// opacity is corrected to 1 - (1 - a)^(2^l)), so coarse levels cost fewer samples.  Kept
// apart so that these template instances compile in parallel with the others.
#include "render_common.cuh"

namespace volrc {
namespace {

template <int DT, int BS, bool Q>
const void* pick_b(bool lod) {
    return lod ? (const void*)k_render<DT, true, kDvr, BS, Q, true> : (const void*)k_render<DT, false, kDvr, BS, Q, true>;
}

template <int DT>
const void* pick_d(int brick, bool quad, bool lod) {
    if (!quad) return pick_b<DT, 0, false>(lod);
    if (brick == 32) return pick_b<DT, 32, true>(lod);
    if (brick == 64) return pick_b<DT, 64, true>(lod);
    return pick_b<DT, 0, true>(lod);
}

}  // namespace

const void* pick_render_level_step(int dtype, int brick, bool quad, bool lod) {
    switch (dtype) {
    case VOL_U8: return pick_d<VOL_U8>(brick, quad, lod);
    case VOL_U16: return pick_d<VOL_U16>(brick, quad, lod);
    case VOL_F16: return pick_d<VOL_F16>(brick, quad, lod);
    case VOL_F32: return pick_d<VOL_F32>(brick, quad, lod);
    }
    return nullptr;
}

}  // namespace volrc
