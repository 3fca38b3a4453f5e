// kernels_sparse.cu -- variants of the forward kernel for volumes addressed through the
// three-level sparse page table (Sec. III-E; the virtual zettabyte volume of Sec. V-C):
// every sample finds its slot through the level's top grid, a middle page and a leaf page.
#include "render_common.cuh"

namespace volrc {
namespace {

template <int DT, int BS, bool Q>
const void* pick_b(bool lod) {
    return lod ? (const void*)k_render<DT, true, kDvr, BS, Q, false, true>
               : (const void*)k_render<DT, false, kDvr, BS, Q, false, true>;
}

template <int DT>
const void* pick_d(int brick, bool quad, bool lod) {
    if (!quad) return pick_b<DT, 0, false>(lod);
    if (brick == 32) return pick_b<DT, 32, true>(lod);
    if (brick == 64) return pick_b<DT, 64, true>(lod);
    return pick_b<DT, 0, true>(lod);
}

}  // namespace

const void* pick_render_sparse(int dtype, int brick, bool quad, bool lod) {
    switch (dtype) {
    case VOL_U8: return pick_d<VOL_U8>(brick, quad, lod);
    case VOL_U16: return pick_d<VOL_U16>(brick, quad, lod);
    case VOL_F16: return pick_d<VOL_F16>(brick, quad, lod);
    case VOL_F32: return pick_d<VOL_F32>(brick, quad, lod);
    }
    return nullptr;
}

}  // namespace volrc
