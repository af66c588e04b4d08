// Shared device-side definitions of the LKS solver: lattice tables, problem geometry, per-step pose.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lks {

// ------------------------------------------------------------------------------------------------
// Velocity sets (Sec. 2.2): D2Q9 for D = 2, D3Q15 for D = 3.  Weights 4/9, 1/9, 1/36 and
// 2/9, 1/9, 1/72.  Functions are constexpr so fully unrolled loops fold every c_i and w_i.
// ------------------------------------------------------------------------------------------------
template <int D>
struct Lattice;

template <>
struct Lattice<2> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int c(int i, int a) {
        // rest, 4 axis velocities, 4 diagonals
        return (i == 0)   ? 0
               : (i == 1) ? (a == 0 ? 1 : 0)
               : (i == 2) ? (a == 1 ? 1 : 0)
               : (i == 3) ? (a == 0 ? -1 : 0)
               : (i == 4) ? (a == 1 ? -1 : 0)
               : (i == 5) ? 1
               : (i == 6) ? (a == 0 ? -1 : 1)
               : (i == 7) ? -1
                          : (a == 0 ? 1 : -1);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <>
struct Lattice<3> {
    static constexpr int Q = 15;
    __host__ __device__ static constexpr int c(int i, int a) {
        // 0: rest; 1..6: +-e_x, +-e_y, +-e_z; 7..14: (+-1, +-1, +-1)
        return (i == 0) ? 0
               : (i <= 6)
                   ? (((i - 1) / 2 == a) ? (((i - 1) % 2 == 0) ? 1 : -1) : 0)
                   : ((((i - 7) >> (2 - a)) & 1) ? -1 : 1);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
};

// Index of the symmetric pair (a, b) in the packed order xx, yy, (zz), xy, (xz, yz).
template <int D>
__host__ __device__ constexpr int sym(int a, int b) {
    return a == b ? a : (D == 2 ? 2 : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)));
}
template <int D>
struct NSym { static constexpr int value = D * (D + 1) / 2; };

// ------------------------------------------------------------------------------------------------
// Problem geometry, passed by value to every kernel.
// ------------------------------------------------------------------------------------------------
struct Geom {
    int n[3];           // analysis grid (n[2] = 1 in 2D)
    int periodic[3];    // 1 periodic, 0 wall planes at 0 and n-1
    long long N;        // number of analysis nodes
    int nde[3];         // design grid including the margin (1 on an unused axis)
    int hw;             // transfer-kernel half width: 1 linear (hat), 2 cosine
    int Fb[3];          // footprint box per axis: nde + 2 hw - 1 (1 on an unused axis)
    long long Fbn;      // footprint box nodes
    int probe_lo[3], probe_hi[3];
    double dir[3];      // objective direction n
    double phi;         // 1 / (Nt |O|): the objective's weight of one node-step
    double phi_var;     // phi of Eq. objective1: weight of the variance V in J1 = E - phi V
    long long jsq_off;  // from an objective slot (sum of n.u) to its twin (sum of (n.u)^2)
    const double* obj;  // device objective terms of the last forward: J, E, V, 1 + 2 phi E
    double A;           // 3/4 - 9 nu / 2
    double wall_u[3][2][3];
    double u_crit2;     // squared stability limit (<= 0 disables)
    int rot;            // 1: the body also rotates (theta turns x-y about an axis parallel to z); the footprint box
                        // on x and y then covers the design grid at any angle (lks_rot.cuh)
    const void* rotmap; // rotating body: kappa, u^S_0 .. u^S_D-1 of the current step on the footprint box (forward)
    unsigned* status;   // device status word of the context (bit 1: a bounded device-side wait expired), or nullptr
    unsigned long long wait_ns;  // limit of one bounded device-side wait in ns (0: one second)
    int wait_probe;     // diagnostic: the plane-pair blocks with tensor copies first wait on a barrier that nothing
                        // completes, so that the wait expires
};

// Per-step rigid-body pose (Eq. rigid_body_position with theta = 0) reduced to what the mapping needs:
// the footprint box origin per axis, the 2 hw tap weights of the shifted design grid and their derivative
// with respect to the offset, and the body velocity u^G.
struct Pose {
    int xs[3];          // footprint box start (folded into [0, n) on periodic axes)
    int pad;
    double w[3][4];     // weight of tap k: design index j = b - 2 hw + 1 + k for box coordinate b
    double dw[3][4];    // d w / d offset
    double uG[3];
    float wf[3][4];     // FP32 copies for the FP32 state path (no FP64 work per node)
    float dwf[3][4];
    float uGf[3];
    float padf;
    // rotating body (Eqs. rigid_body_position, rigid_body_velocity): theta, omega, (cos, sin) theta, and x^G - xs on
    // x and y (the rotation centre relative to the footprint box start); theta = 0 without rotation
    double th, om, cs[2], cg[2];
    float thf, omf, csf[2], cgf[2];
};

// Pose values in the state precision T.
template <typename T>
__device__ __forceinline__ T pose_w(const Pose& P, int a, int k);
template <>
__device__ __forceinline__ double pose_w<double>(const Pose& P, int a, int k) { return P.w[a][k]; }
template <>
__device__ __forceinline__ float pose_w<float>(const Pose& P, int a, int k) { return P.wf[a][k]; }
template <typename T>
__device__ __forceinline__ T pose_dw(const Pose& P, int a, int k);
template <>
__device__ __forceinline__ double pose_dw<double>(const Pose& P, int a, int k) { return P.dw[a][k]; }
template <>
__device__ __forceinline__ float pose_dw<float>(const Pose& P, int a, int k) { return P.dwf[a][k]; }
template <typename T>
__device__ __forceinline__ T pose_uG(const Pose& P, int a);
template <>
__device__ __forceinline__ double pose_uG<double>(const Pose& P, int a) { return P.uG[a]; }
template <>
__device__ __forceinline__ float pose_uG<float>(const Pose& P, int a) { return P.uGf[a]; }

// Periodic wrap (no integer division: halo indices are at most a tile past the grid, so the loops run
// zero or one time except on grids smaller than a tile).
__host__ __device__ inline int wrap(int x, int n) {
    while (x < 0) x += n;
    while (x >= n) x -= n;
    return x;
}

// Box coordinate of analysis coordinate x along one axis, or -1 when x is outside the footprint box.
__device__ __forceinline__ int box_coord(int x, int xs, int Fb, int n, int periodic) {
    int b = x - xs;
    if (periodic && b < 0) b += n;
    return (b >= 0 && b < Fb) ? b : -1;
}

}  // namespace lks
