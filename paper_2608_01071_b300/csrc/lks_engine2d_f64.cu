// Engine2D<double> instantiations (one translation unit per lattice and precision, compiled in parallel).
#include "lks_engine2d.cuh"

namespace lks {

Engine* make_engine2d_f64(int hw, const Geom& g) {
    return hw == 1 ? (Engine*)new Engine2D<double, 1>(g) : (Engine*)new Engine2D<double, 2>(g);
}

}  // namespace lks
