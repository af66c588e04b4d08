// Objective J2 of Eq. objective2 (the oar) for a rotating body: F_L + w_D F_D + w_T T with the torque term, and its
// adjoint pieces.
//
// With rotation the design-grid integrals are taken on the design grid itself, as the equation states: per step n and
// design node j,
//   r_j = R(theta)(xi_j - xi^G)                          (the arm, x-y; Eq. rigid_body_position),
//   U_j = sum_x W(x - x^ref_j) u_n(x)                    (u^ref: the velocity interpolated at x^ref_j = r_j + x^G),
//   v_j = u^G + omega J r_j,  J r = (-r_y, r_x)           (u^S,ref of Eq. rigid_body_velocity),
//   F_j = kappa^ref_j (U_j - v_j)                        (the Brinkman force density),
//   F_L = c_L sum_j F_j,x,  w_D F_D = c_D u^G_y sum_j F_j,y,  w_T T = c_T omega sum_j (r_j,x F_j,y - r_j,y F_j,x),
// with c_L = 1 / (Nt |D|), c_D = w_D / (drag_span |D|), c_T = w_T / (2 pi l_m |D|) (the margin has kappa^ref = 0, so
// the sums may run over the extended grid).  With g_j = (c_L - c_T omega r_j,y, c_D u^G_y + c_T omega r_j,x) the
// partial derivatives of j2_n are
//   d/du_n(x)          = sum_j W(x - x^ref_j) kappa^ref_j g_j        (the adjoint source, on the analysis grid),
//   d/dkappa^ref_j     = g_j . (U_j - v_j),
//   d/do (= d/dx^G)    = sum_j gx_j,   gx_j,a = sum_b kappa^ref_j g_j,b dU_j,b/dx^ref_a,
//   d/du^G             = (-c_L K + c_T omega (R M1)_y,  -c_D u^G_y K - c_T omega (R M1)_x + c_D sum_j F_j,y),
//   d/domega           = c_L (R M1)_y - c_D u^G_y (R M1)_x - c_T omega I + c_T sum_j r_j x F_j,
//   d/dtheta           = omega (c_L (R M1)_x + c_D u^G_y (R M1)_y) + sum_j gx_j . J r_j - c_T omega sum_j r_j . F_j,
// where K = sum_j kappa^ref_j, M1 = sum_j kappa^ref_j (xi_j - xi^G) and I = sum_j kappa^ref_j |xi_j - xi^G|^2 do
// not change with the step.  Everything but the adjoint source depends on the forward state only, so the forward
// sweep accumulates it: the per-step sums (oar_rot_partial_kernel) and d/dkappa^ref summed over the steps per design
// node (a Kahan-compensated sum in the state precision: the FP64 pipe of this part is too narrow for an FP64
// addition per design node and step).
#pragma once

#include "lks_oar.cuh"
#include "lks_rot.cuh"

namespace lks {

constexpr int kOarRotNV = 8;  // per-step sums: F_x, F_y, sum r x F, sum r . F, gx (3), gx . J r

// Per-step sums of one step on the design side (slot[kOarRotNV], by the last block) and the compensated per-node
// accumulation of d j2_n / d kappa^ref_j (kh - kl).  st is the state of step n.
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) oar_rot_partial_kernel(Geom g, OarGeom o, const Pose* __restrict__ pose,
                                                              const T* __restrict__ kref, const T* __restrict__ st,
                                                              T* __restrict__ kh, T* __restrict__ kl,
                                                              double* __restrict__ scratch, unsigned* __restrict__ ticket,
                                                              double* __restrict__ slot) {
    constexpr int NV = kOarRotNV;
    __shared__ double red[NV * 8];
    const Pose& P = *pose;
    const int nde0 = g.nde[0], nde1 = g.nde[1];
    const int nd = nde0 * nde1 * g.nde[2];
    const int jl = blockIdx.x * 256 + threadIdx.x;
    T v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0;
    if (jl < nd) {
        const int jx = jl % nde0, jy = (jl / nde0) % nde1, jz = jl / (nde0 * nde1);
        const T c = pose_cos<T>(P), s = pose_sin<T>(P), om = pose_om<T>(P);
        const T ax = (T)jx - (T)(0.5 * (nde0 - 1)), ay = (T)jy - (T)(0.5 * (nde1 - 1));
        const T rx = c * ax - s * ay, ry = s * ax + c * ay;
        // x^ref in footprint-box coordinates: x-y from the rotation about x^G, z from the translation taps
        const T qx = pose_cg<T>(P, 0) + rx, qy = pose_cg<T>(P, 1) + ry;
        T U[3] = {0, 0, 0}, dU[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // dU[a][b] = dU_b / dx^ref_a
        const int bx0 = (int)ceil(qx - (T)HW), bx1 = (int)floor(qx + (T)HW);
        const int by0 = (int)ceil(qy - (T)HW), by1 = (int)floor(qy + (T)HW);
#pragma unroll
        for (int k = 0; k < (D == 3 ? 2 * HW : 1); ++k) {
            const int bz = D == 3 ? jz + 2 * HW - 1 - k : 0;
            const T wz = D == 3 ? pose_w<T>(P, 2, k) : (T)1, dwz = D == 3 ? pose_dw<T>(P, 2, k) : (T)0;
            if (wz == (T)0 && dwz == (T)0) continue;
            int xz = 0;
            if (D == 3) {
                xz = P.xs[2] + bz;
                if (g.periodic[2]) {
                    if (xz >= g.n[2]) xz -= g.n[2];
                } else if (xz < 0 || xz >= g.n[2]) {
                    continue;
                }
            }
            for (int by = by0; by <= by1; ++by) {
                T wy, dwy;
                rot_w<T, HW>((T)by - qy, wy, dwy);
                int yy = P.xs[1] + by;
                if (g.periodic[1]) {
                    if (yy >= g.n[1]) yy -= g.n[1];
                } else if (yy < 0 || yy >= g.n[1]) {
                    continue;
                }
                for (int bx = bx0; bx <= bx1; ++bx) {
                    T wx, dwx;
                    rot_w<T, HW>((T)bx - qx, wx, dwx);
                    int xx = P.xs[0] + bx;
                    if (g.periodic[0]) {
                        if (xx >= g.n[0]) xx -= g.n[0];
                    } else if (xx < 0 || xx >= g.n[0]) {
                        continue;
                    }
                    const long long gi = xx + (long long)g.n[0] * (yy + (long long)g.n[1] * xz);
                    const T W = wx * wy * wz;
                    const T Wa[3] = {dwx * wy * wz, wx * dwy * wz, wx * wy * dwz};
#pragma unroll
                    for (int b = 0; b < D; ++b) {
                        const T ub = st[(1 + b) * g.N + gi];
                        U[b] += W * ub;
#pragma unroll
                        for (int a = 0; a < D; ++a) dU[a][b] += Wa[a] * ub;
                    }
                }
            }
        }
        const T uGx = pose_uG<T>(P, 0), uGy = pose_uG<T>(P, 1);
        const T kr = kref[jl];
        const T ex = U[0] - (uGx - om * ry), ey = U[1] - (uGy + om * rx);  // U - v (x-y)
        const T Fx = kr * ex, Fy = kr * ey;
        const T gxw = (T)o.cL - (T)o.cT * om * ry, gyw = (T)(o.cD) * uGy + (T)o.cT * om * rx;
        // d j2_n / d kappa^ref_j, compensated running sum over the steps
        {
            const T y = (gxw * ex + gyw * ey) - kl[jl];
            const T t = kh[jl] + y;
            kl[jl] = (t - kh[jl]) - y;
            kh[jl] = t;
        }
        v[0] = Fx;
        v[1] = Fy;
        v[2] = rx * Fy - ry * Fx;
        v[3] = rx * Fx + ry * Fy;
        T gx[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) gx[a] = kr * (gxw * dU[a][0] + gyw * dU[a][1]);
        v[4] = gx[0];
        v[5] = gx[1];
        v[6] = gx[2];
        v[7] = gx[0] * -ry + gx[1] * rx;
    }
    double out[NV];
    block_sum<256, NV, T>(v, out, red);
    last_block_sum<NV>(out, scratch, ticket, (int)gridDim.x, slot, red);
}

// K, M1 (x-y) and I of the current kappa^ref (FP64, extended grid) into cst[4]: per-block partials, summed by the
// last block.
static __global__ void __launch_bounds__(256) oar_rot_const_kernel(const double* __restrict__ kref64, int nde0,
                                                                   int nde1, int nde2, double* __restrict__ scratch,
                                                                   unsigned* __restrict__ ticket,
                                                                   double* __restrict__ cst) {
    __shared__ double red[4 * 8];
    const long long nd = (long long)nde0 * nde1 * nde2;
    const long long jl = blockIdx.x * 256LL + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (jl < nd) {
        const int jx = (int)(jl % nde0), jy = (int)((jl / nde0) % nde1);
        const double ax = jx - 0.5 * (nde0 - 1), ay = jy - 0.5 * (nde1 - 1), k = kref64[jl];
        v[0] = k;
        v[1] = k * ax;
        v[2] = k * ay;
        v[3] = k * (ax * ax + ay * ay);
    }
    double out[4];
    block_sum<256, 4, double>(v, out, red);
    last_block_sum<4>(out, scratch, ticket, (int)gridDim.x, cst, red);
}

// J2 from the per-step sums (obj[0]) and the per-step explicit derivatives (one block; fixed reduction order):
// go[n][D] (position), guG[n][D], gth[n], gom[n].
static __global__ void oar_rot_reduce_kernel(OarGeom og, const double* __restrict__ slot, int Nt,
                                             const Pose* __restrict__ poses, const double* __restrict__ cst, int D,
                                             double* __restrict__ obj, double* __restrict__ go,
                                             double* __restrict__ guG, double* __restrict__ gth,
                                             double* __restrict__ gom) {
    __shared__ double red[32];
    const int tid = threadIdx.x, nw = (blockDim.x + 31) / 32;
    const double K = cst[0], M1x = cst[1], M1y = cst[2], I = cst[3], cL = og.cL, cD = og.cD, cT = og.cT;
    double tot = 0.0;
    for (int n = 1 + tid; n <= Nt; n += blockDim.x) {
        const double* sl = slot + (long long)n * kOarRotNV;
        const Pose& P = poses[n];
        const double c = P.cs[0], s = P.cs[1], om = P.om, uy = P.uG[1];
        const double RMx = c * M1x - s * M1y, RMy = s * M1x + c * M1y;
        const double Fx = sl[0], Fy = sl[1], Tq = sl[2], rF = sl[3], gxJr = sl[7];
        tot += cL * Fx + cD * uy * Fy + cT * om * Tq;
        for (int a = 0; a < D; ++a) {
            go[(long long)n * D + a] = sl[4 + a];
            guG[(long long)n * D + a] = a == 0 ? -cL * K + cT * om * RMy
                                               : (a == 1 ? -cD * uy * K - cT * om * RMx + cD * Fy : 0.0);
        }
        gom[n] = cL * RMy - cD * uy * RMx - cT * om * I + cT * Tq;
        gth[n] = om * (cL * RMx + cD * uy * RMy) + gxJr - cT * om * rF;
    }
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < nw; ++i) sum += red[i];
        obj[0] = sum;
    }
}

// Adjoint source of step n on the fluid nodes of the footprint box: lambda_u += sum_j W(x - x^ref_j) kappa^ref_j g_j,
// i.e. (c_L kappa - c_T omega kappa_r,y, c_D u^G_y kappa + c_T omega kappa_r,x) with kappa_r = sum_j W kappa^ref_j r_j
// (the rotated gather of rot_sums, with kappa^ref-weighted arms).
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) oar_rot_source_kernel(Geom g, OarGeom o, const Pose* __restrict__ pose,
                                                             const T* __restrict__ kref, T* __restrict__ lam) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    const Pose& P = *pose;
    int b[3] = {0, 0, 0};
    const long long gi = rot_box_node<D>(g, P, bl, b);
    if (gi < 0) return;
    int x[3] = {(int)(gi % g.n[0]), (int)((gi / g.n[0]) % g.n[1]), (int)(gi / ((long long)g.n[0] * g.n[1]))};
    T uw[D];
    if (wall_node<T, D>(g, x, uw)) return;
    const T c = pose_cos<T>(P), s = pose_sin<T>(P), om = pose_om<T>(P);
    const T gx = (T)(0.5 * (g.nde[0] - 1)), gy = (T)(0.5 * (g.nde[1] - 1));
    const T px = (T)b[0] - pose_cg<T>(P, 0), py = (T)b[1] - pose_cg<T>(P, 1);
    const T qx = c * px + s * py + gx, qy = -s * px + c * py + gy;
    const T reach = (T)(1.4142135623730951 * HW + 1e-4);
    const int jx0 = max(0, (int)ceil(qx - reach)), jx1 = min(g.nde[0] - 1, (int)floor(qx + reach));
    const int jy0 = max(0, (int)ceil(qy - reach)), jy1 = min(g.nde[1] - 1, (int)floor(qy + reach));
    T wz[2 * HW];
    int jz[2 * HW];
#pragma unroll
    for (int k = 0; k < 2 * HW; ++k) {
        jz[k] = D == 3 ? b[D - 1] - 2 * HW + 1 + k : 0;
        const bool v = D == 2 || (jz[k] >= 0 && jz[k] < g.nde[2]);
        wz[k] = D == 2 ? (k == 0 ? (T)1 : (T)0) : (v ? pose_w<T>(P, 2, k) : (T)0);
    }
    const long long sxy = (long long)g.nde[0] * g.nde[1];
    T K0 = 0, KAx = 0, KAy = 0;  // sum_j W kappa^ref_j (1, arm_x, arm_y)
    for (int jy = jy0; jy <= jy1; ++jy) {
        const T ay = (T)jy - gy;
        for (int jx = jx0; jx <= jx1; ++jx) {
            const T ax = (T)jx - gx;
            const T rx = px - (c * ax - s * ay), ry = py - (s * ax + c * ay);
            T wx, dwx, wy, dwy;
            rot_w<T, HW>(rx, wx, dwx);
            rot_w<T, HW>(ry, wy, dwy);
            const T W = wx * wy;
            if (W == (T)0) continue;
            T kr = 0;
            const long long jbase = jx + (long long)g.nde[0] * jy;
#pragma unroll
            for (int k = 0; k < 2 * HW; ++k) {
                if (D == 2 && k > 0) break;
                if (wz[k] == (T)0) continue;
                kr += wz[k] * kref[jbase + sxy * (D == 3 ? jz[k] : 0)];
            }
            K0 += W * kr;
            KAx += W * kr * ax;
            KAy += W * kr * ay;
        }
    }
    const T Krx = c * KAx - s * KAy, Kry = s * KAx + c * KAy;  // kappa_r = R(theta) sum W kappa^ref arm
    lam[g.N + gi] += (T)o.cL * K0 - (T)o.cT * om * Kry;
    lam[2 * g.N + gi] += (T)o.cD * pose_uG<T>(P, 1) * K0 + (T)o.cT * om * Krx;
}

// The explicit terms of the rotating body's J2 into the reverse sweep's gradients: dJ/ds_n += go[n],
// dJ/du^G_n += guG[n], dJ/dtheta_n += gth[n], dJ/domega_n += gom[n] (n >= 1), and dJ/dkappa^ref_j += kh_j - kl_j.
template <typename T>
__global__ void oar_rot_apply_kernel(int Nt, int D, const double* __restrict__ go, const double* __restrict__ guG,
                                     const double* __restrict__ gth, const double* __restrict__ gom,
                                     const T* __restrict__ kh, const T* __restrict__ kl, double* __restrict__ g_s,
                                     double* __restrict__ g_uG, double* __restrict__ g_th, double* __restrict__ g_om,
                                     double* __restrict__ dkref, long long nde) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nde) dkref[i] += (double)kh[i] - (double)kl[i];  // the compensation kl holds the lost part, negated
    if (i >= 1 && i <= Nt) {
        for (int c = 0; c < D; ++c) {
            g_s[i * D + c] += go[i * D + c];
            g_uG[i * D + c] += guG[i * D + c];
        }
        g_th[i] += gth[i];
        g_om[i] += gom[i];
    }
}

}  // namespace lks
