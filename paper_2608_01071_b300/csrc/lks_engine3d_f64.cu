// Engine3D<double> instantiations (one translation unit per lattice and precision, compiled in parallel).
#include "lks_engine3d.cuh"

namespace lks {

Engine* make_engine3d_f64(int hw, const Geom& g) {
    return hw == 1 ? (Engine*)new Engine3D<double, 1>(g) : (Engine*)new Engine3D<double, 2>(g);
}

}  // namespace lks
