// Engine3D<float> instantiations (one translation unit per lattice and precision, compiled in parallel).
#include "lks_engine3d.cuh"

namespace lks {

Engine* make_engine3d_f32(int hw, const Geom& g) {
    return hw == 1 ? (Engine*)new Engine3D<float, 1>(g) : (Engine*)new Engine3D<float, 2>(g);
}

}  // namespace lks
