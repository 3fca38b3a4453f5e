// kernels_skip.cu -- variants of the forward kernel with empty-space skipping (the paper's
// empty-space skipping: the table of uniform chunks of Sec. III-H and the ES column of Sec. IV-A) for
// emission/absorption compositing.  A sample in a
// brick or 8^3-cell block whose value range the transfer function maps to zero opacity jumps
// to the end of the run of such blocks; the image does not change.
#include "render_common.cuh"

namespace volrc {
namespace {

template <int DT, int BS, bool Q, int MODE>
const void* pick_b(bool lod) {
    return lod ? (const void*)k_render<DT, true, MODE, BS, Q, false, false, true>
               : (const void*)k_render<DT, false, MODE, BS, Q, false, false, true>;
}

template <int DT, int MODE>
const void* pick_d(int brick, bool quad, bool lod) {
    if (!quad) return pick_b<DT, 0, false, MODE>(lod);
    if (brick == 32) return pick_b<DT, 32, true, MODE>(lod);
    if (brick == 64) return pick_b<DT, 64, true, MODE>(lod);
    return nullptr;
}

template <int MODE>
const void* pick_m(int dtype, int brick, bool quad, bool lod) {
    switch (dtype) {
    case VOL_U8: return pick_d<VOL_U8, MODE>(brick, quad, lod);
    case VOL_U16: return pick_d<VOL_U16, MODE>(brick, quad, lod);
    case VOL_F16: return pick_d<VOL_F16, MODE>(brick, quad, lod);
    case VOL_F32: return pick_d<VOL_F32, MODE>(brick, quad, lod);
    }
    return nullptr;
}

}  // namespace

const void* pick_render_skip(int dtype, int brick, bool quad, bool lod, int mode) {
    // (gradient mode renders without skipping: the adjoint reads a value for every sample)
    if (mode == kDvr) return pick_m<kDvr>(dtype, brick, quad, lod);
    return nullptr;
}

}  // namespace volrc
