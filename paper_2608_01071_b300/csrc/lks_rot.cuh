// Rigidly rotating body: the mapping of Eqs. kappa and u_s for a pose with theta != 0 (Sec. 2.3, Eqs.
// rigid_body_position x^ref_j = R(theta)(xi_j - xi^G) + x^G and rigid_body_velocity u^S,ref_j = R'(theta)(xi_j - xi^G)
// omega + u^G; theta turns the x-y components about an axis parallel to z), its derivatives with respect to the
// position, theta and omega (Sec. 2.5, Eq. dJdpsi), and the transposed mapping on the design side.
//
// The rotated design lattice is not aligned with the analysis axes, so the tap product of the translation case holds
// only along z.  A node of the footprint box at position p relative to x^G (x-y) gathers from the design nodes j
// whose arms R(theta)(xi_j - xi^G) lie within the kernel's support around p: their arms lie inside the square of half
// width hw turned back by -theta, so the candidates are the design nodes within hw sqrt(2) of R(-theta) p + xi^G per
// axis (3 x 3 for the hat, 6 x 6 for the cosine kernel).  Along z the taps are those of the translation (pose.w[2]).
// The footprint box is fixed per problem: on x and y it covers the design grid's circumscribed circle plus the
// kernel's half width around x^G (pose.cg: x^G relative to the box start); on z it is the translation box.
//
// Weights follow the transfer kernel w and its derivative with the tap-piece convention of the translation taps
// (for the hat w'(r) = -1 on (0, 1] and +1 on (-1, 0]); dW/dx^ref = -w'(r).
#pragma once

#include "lks_step_kernels.cuh"

namespace lks {

template <typename T, int HW>
__device__ __forceinline__ void rot_w(T r, T& w, T& dw) {
    if (HW == 1) {
        const T ar = r < (T)0 ? -r : r;
        w = ar <= (T)1 ? (T)1 - ar : (T)0;
        dw = (r > (T)0 && r <= (T)1) ? (T)1 : ((r > (T)-1 && r <= (T)0) ? (T)-1 : (T)0);
    } else {
        const bool in = (r < (T)0 ? -r : r) <= (T)2;
        const double h = 0.5 * (double)r;
        w = in ? (T)(0.25 * (1.0 + cospi(h))) : (T)0;
        dw = in ? (T)(0.39269908169872414 * sinpi(h)) : (T)0;  // pi/8 sin(pi r / 2)
    }
}

template <typename T>
__device__ __forceinline__ T pose_cos(const Pose& P);
template <>
__device__ __forceinline__ double pose_cos<double>(const Pose& P) { return P.cs[0]; }
template <>
__device__ __forceinline__ float pose_cos<float>(const Pose& P) { return P.csf[0]; }
template <typename T>
__device__ __forceinline__ T pose_sin(const Pose& P);
template <>
__device__ __forceinline__ double pose_sin<double>(const Pose& P) { return P.cs[1]; }
template <>
__device__ __forceinline__ float pose_sin<float>(const Pose& P) { return P.csf[1]; }
template <typename T>
__device__ __forceinline__ T pose_cg(const Pose& P, int a);
template <>
__device__ __forceinline__ double pose_cg<double>(const Pose& P, int a) { return P.cg[a]; }
template <>
__device__ __forceinline__ float pose_cg<float>(const Pose& P, int a) { return P.cgf[a]; }
template <typename T>
__device__ __forceinline__ T pose_om(const Pose& P);
template <>
__device__ __forceinline__ double pose_om<double>(const Pose& P) { return P.om; }
template <>
__device__ __forceinline__ float pose_om<float>(const Pose& P) { return P.omf; }

// Sums of the rotated mapping at one node of the footprint box: kappa = sum_j W kappa^ref_j, C = sum_j W,
// A = sum_j W arm_j (x-y arms), and with GRAD their derivatives with respect to x^ref (the position o) and theta.
template <typename T, int D>
struct RotSums {
    T kap, C, A[2];
    T dk[D], dkth, dC[D], dCth, dA[D][2], dAth[2];
};

template <typename T, int D, int HW, bool GRAD>
__device__ __forceinline__ void rot_sums(const Geom& g, const Pose& P, const T* __restrict__ kref, const int* b,
                                         RotSums<T, D>& S) {
    const T c = pose_cos<T>(P), s = pose_sin<T>(P);
    const T gx = (T)(0.5 * (g.nde[0] - 1)), gy = (T)(0.5 * (g.nde[1] - 1));
    // node relative to x^G, and the same point in design coordinates (turned back by -theta, shifted by xi^G)
    const T px = (T)b[0] - pose_cg<T>(P, 0), py = (T)b[1] - pose_cg<T>(P, 1);
    const T qx = c * px + s * py + gx, qy = -s * px + c * py + gy;
    const T reach = (T)(1.4142135623730951 * HW + 1e-4);
    const int jx0 = max(0, (int)ceil(qx - reach)), jx1 = min(g.nde[0] - 1, (int)floor(qx + reach));
    const int jy0 = max(0, (int)ceil(qy - reach)), jy1 = min(g.nde[1] - 1, (int)floor(qy + reach));
    S.kap = S.C = S.A[0] = S.A[1] = 0;
    if (GRAD) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            S.dk[a] = S.dC[a] = S.dA[a][0] = S.dA[a][1] = 0;
        }
        S.dkth = S.dCth = S.dAth[0] = S.dAth[1] = 0;
    }
    // z taps (translation): design plane jz = b_z - 2 hw + 1 + k with weight pose.w[2][k]
    T wz[2 * HW], dwz[2 * HW];
    int jz[2 * HW];
    T szw = 0, szd = 0;
#pragma unroll
    for (int k = 0; k < 2 * HW; ++k) {
        jz[k] = D == 3 ? b[D - 1] - 2 * HW + 1 + k : 0;
        const bool v = D == 2 || (jz[k] >= 0 && jz[k] < g.nde[2]);
        wz[k] = D == 2 ? (k == 0 ? (T)1 : (T)0) : (v ? pose_w<T>(P, 2, k) : (T)0);
        dwz[k] = D == 2 ? (T)0 : (v ? pose_dw<T>(P, 2, k) : (T)0);
        szw += wz[k];
        szd += dwz[k];
    }
    const long long sxy = (long long)g.nde[0] * g.nde[1];
    for (int jy = jy0; jy <= jy1; ++jy) {
        const T ay = (T)jy - gy;
        for (int jx = jx0; jx <= jx1; ++jx) {
            const T ax = (T)jx - gx;
            // x^ref - x^G = R arm; r = p - R arm
            const T rx = px - (c * ax - s * ay), ry = py - (s * ax + c * ay);
            T wx, dwx, wy, dwy;
            rot_w<T, HW>(rx, wx, dwx);
            rot_w<T, HW>(ry, wy, dwy);
            const T W = wx * wy;
            const T Wx = dwx * wy, Wy = wx * dwy;  // dW/dx^ref_x, dW/dx^ref_y
            if (W == (T)0 && (!GRAD || (Wx == (T)0 && Wy == (T)0))) continue;
            // d x^ref / d theta = R' arm
            const T tx = -s * ax - c * ay, ty = c * ax - s * ay;
            const T Wth = Wx * tx + Wy * ty;
            T kr = 0;
            T dkz = 0;
            const long long jbase = jx + (long long)g.nde[0] * jy;
#pragma unroll
            for (int k = 0; k < 2 * HW; ++k) {
                if (D == 2 && k > 0) break;
                if (wz[k] == (T)0 && dwz[k] == (T)0) continue;
                const T kv = kref[jbase + sxy * (D == 3 ? jz[k] : 0)];
                kr += wz[k] * kv;
                dkz += dwz[k] * kv;
            }
            S.kap += W * kr;
            S.C += W * szw;
            S.A[0] += W * szw * ax;
            S.A[1] += W * szw * ay;
            if (GRAD) {
                S.dk[0] += Wx * kr;
                S.dk[1] += Wy * kr;
                S.dkth += Wth * kr;
                S.dC[0] += Wx * szw;
                S.dC[1] += Wy * szw;
                S.dCth += Wth * szw;
                S.dA[0][0] += Wx * szw * ax;
                S.dA[0][1] += Wx * szw * ay;
                S.dA[1][0] += Wy * szw * ax;
                S.dA[1][1] += Wy * szw * ay;
                S.dAth[0] += Wth * szw * ax;
                S.dAth[1] += Wth * szw * ay;
                if (D == 3) {
                    S.dk[D - 1] += W * dkz;
                    S.dC[D - 1] += W * szd;
                    S.dA[D - 1][0] += W * szd * ax;
                    S.dA[D - 1][1] += W * szd * ay;
                }
            }
        }
    }
}

// u^S = C u^G + omega R'(theta) A on x-y, C u^G_z on z (Eq. rigid_body_velocity mapped by Eq. u_s)
template <typename T, int D>
__device__ __forceinline__ void rot_uS(const Pose& P, const RotSums<T, D>& S, T* uS) {
    const T c = pose_cos<T>(P), s = pose_sin<T>(P), om = pose_om<T>(P);
    uS[0] = S.C * pose_uG<T>(P, 0) + om * (-s * S.A[0] - c * S.A[1]);
    uS[1] = S.C * pose_uG<T>(P, 1) + om * (c * S.A[0] - s * S.A[1]);
    if (D == 3) uS[D - 1] = S.C * pose_uG<T>(P, D - 1);
}

// Box node bl -> box coordinates b and the analysis node index (-1 outside the grid on a wall axis).
template <int D>
__device__ __forceinline__ long long rot_box_node(const Geom& g, const Pose& P, long long bl, int* b) {
    long long gi = 0, stride = 1;
    box_unflatten<D>(g, bl, b);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int v = P.xs[a] + b[a];
        if (g.periodic[a]) {
            if (v >= g.n[a]) v -= g.n[a];
        } else if (v < 0 || v >= g.n[a]) {
            return -1;
        }
        gi += v * stride;
        stride *= g.n[a];
    }
    return gi;
}

// kappa and u^S of one step on the footprint box, for the forward step: map[(1 + D) Fbn] = kappa, u^S_0 .. u^S_D-1.
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) rot_box_map_kernel(Geom g, const Pose* __restrict__ pose,
                                                          const T* __restrict__ kref, T* __restrict__ map) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    int b[3] = {0, 0, 0};
    rot_box_node<D>(g, *pose, bl, b);
    RotSums<T, D> S;
    rot_sums<T, D, HW, false>(g, *pose, kref, b, S);
    T uS[3];
    rot_uS<T, D>(*pose, S, uS);
    map[bl] = S.kap;
#pragma unroll
    for (int c = 0; c < D; ++c) map[(1 + c) * g.Fbn + bl] = uS[c];
}

// 1 / (1 + kappa) on the footprint box for steps n_first .. n_first + gridDim.y - 1 (stride Fbn per step).
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) rot_box_fac_kernel(Geom g, const Pose* __restrict__ poses,
                                                          const T* __restrict__ kref, int n_first, T* __restrict__ fac) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    const int j = blockIdx.y;
    const Pose& P = poses[n_first + j];
    int b[3] = {0, 0, 0};
    rot_box_node<D>(g, P, bl, b);
    RotSums<T, D> S;
    rot_sums<T, D, HW, false>(g, P, kref, b, S);
    fac[j * g.Fbn + bl] = (T)1 / ((T)1 + S.kap);
}

// Local sensitivities of a segment's steps (b3 with b5 for the rotating body), one box node per thread and step:
//   kappa-bar = lam_u . (u^S - u_n) / (1 + kappa),  u^S-bar = lam_u kappa / (1 + kappa)   (0 off the grid; the records
//   hold lam_u = 0 on walls), written to kbar[step][1 + D][Fbn] for the transposed mapping; per block the step's
//   dJ/do_a, dJ/du^G_a, dJ/dtheta, dJ/domega into mslot[step][block][2 D + 2].
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) rot_sens_kernel(Geom g, const Pose* __restrict__ poses, const T* __restrict__ kref,
                                                       const T* __restrict__ boxbuf, long long bstride, int n_first,
                                                       T* __restrict__ kbar, double* __restrict__ mslot) {
    constexpr int NV = 2 * D + 2;
    __shared__ double red[NV * 8];
    const int st = blockIdx.y;
    const Pose& P = poses[n_first + st];
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    T mv[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) mv[q] = 0;
    if (bl < g.Fbn) {
        int b[3] = {0, 0, 0};
        const long long gi = rot_box_node<D>(g, P, bl, b);
        T kb = 0, ub[3] = {0, 0, 0};
        if (gi >= 0) {
            const T* bb = boxbuf + (long long)st * bstride;
            RotSums<T, D> S;
            rot_sums<T, D, HW, true>(g, P, kref, b, S);
            T uS[3];
            rot_uS<T, D>(P, S, uS);
            const T inv = (T)1 / ((T)1 + S.kap);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const T lu = bb[c * g.Fbn + bl];
                kb += lu * (uS[c] - bb[(D + c) * g.Fbn + bl]);
                ub[c] = lu * S.kap * inv;
            }
            kb *= inv;
            const T cs = pose_cos<T>(P), sn = pose_sin<T>(P), om = pose_om<T>(P);
            const T uG[3] = {pose_uG<T>(P, 0), pose_uG<T>(P, 1), D == 3 ? pose_uG<T>(P, D - 1) : (T)0};
            // dJ/do_a = kappa-bar dkappa/do_a + u^S-bar . du^S/do_a
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T dux = S.dC[a] * uG[0] + om * (-sn * S.dA[a][0] - cs * S.dA[a][1]);
                const T duy = S.dC[a] * uG[1] + om * (cs * S.dA[a][0] - sn * S.dA[a][1]);
                T v = kb * S.dk[a] + ub[0] * dux + ub[1] * duy;
                if (D == 3) v += ub[D - 1] * S.dC[a] * uG[D - 1];
                mv[a] = v;
                mv[D + a] = ub[a] * S.C;  // dJ/du^G_a
            }
            // dJ/dtheta: d u^S / d theta = (dC/dtheta) u^G + omega (R' dA/dtheta + R'' A)
            const T dtx = S.dCth * uG[0] + om * ((-sn * S.dAth[0] - cs * S.dAth[1]) + (-cs * S.A[0] + sn * S.A[1]));
            const T dty = S.dCth * uG[1] + om * ((cs * S.dAth[0] - sn * S.dAth[1]) + (-sn * S.A[0] - cs * S.A[1]));
            T vth = kb * S.dkth + ub[0] * dtx + ub[1] * dty;
            if (D == 3) vth += ub[D - 1] * S.dCth * uG[D - 1];
            mv[2 * D] = vth;
            // dJ/domega: d u^S / d omega = R' A
            mv[2 * D + 1] = ub[0] * (-sn * S.A[0] - cs * S.A[1]) + ub[1] * (cs * S.A[0] - sn * S.A[1]);
        }
        T* kbs = kbar + (long long)st * (1 + D) * g.Fbn;
        kbs[bl] = kb;
#pragma unroll
        for (int c = 0; c < D; ++c) kbs[(1 + c) * g.Fbn + bl] = ub[c];
    }
    double out[NV];
    block_sum<256, NV, T>(mv, out, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) mslot[((long long)st * gridDim.x + blockIdx.x) * NV + q] = out[q];
    }
}

// Transposed mapping on the design side (b4): dJ/dkappa^ref_j += sum_x W(x, x^ref_j(n)) kappa-bar_n(x), over the
// steps of a segment (fixed summation order, no atomics).  The nodes x around x^ref_j are the 2 hw taps per
// axis in box coordinates: x-y around cg + R arm_j, z the translation taps.
template <typename T, int D, int HW>
__global__ void rot_gather_kernel(Geom g, const Pose* __restrict__ poses, const T* __restrict__ kbar, int n_first,
                                  int nsteps, long long kstride, double* __restrict__ dkref) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nde = (long long)g.nde[0] * g.nde[1] * g.nde[2];
    if (j >= nde) return;
    const int jx = (int)(j % g.nde[0]), jy = (int)((j / g.nde[0]) % g.nde[1]), jz = (int)(j / ((long long)g.nde[0] * g.nde[1]));
    const T ax = (T)jx - (T)(0.5 * (g.nde[0] - 1)), ay = (T)jy - (T)(0.5 * (g.nde[1] - 1));
    // running FP64 sum in strict step order n = Nt..1 across calls, as in design_gather_kernel, so that the
    // segmentation of the reverse sweep cannot change the rounding
    double acc = dkref[j];
    for (int st = nsteps - 1; st >= 0; --st) {
        const Pose& P = poses[n_first + st];
        const T c = pose_cos<T>(P), s = pose_sin<T>(P);
        const T cx = pose_cg<T>(P, 0) + (c * ax - s * ay), cy = pose_cg<T>(P, 1) + (s * ax + c * ay);
        const int bx0 = (int)floor(cx) - HW + 1, by0 = (int)floor(cy) - HW + 1;
        const T* kb = kbar + (long long)st * kstride;
        T sum = 0;
#pragma unroll
        for (int kz = 0; kz < (D == 3 ? 2 * HW : 1); ++kz) {
            int bz = 0;
            T wz = 1;
            if (D == 3) {
                bz = jz + 2 * HW - 1 - kz;
                if (bz < 0 || bz >= g.Fb[2]) continue;
                wz = pose_w<T>(P, 2, kz);
            }
#pragma unroll
            for (int ty = 0; ty < 2 * HW; ++ty) {
                const int by = by0 + ty;
                if (by < 0 || by >= g.Fb[1]) continue;
                T wy, dwy;
                rot_w<T, HW>((T)by - cy, wy, dwy);
#pragma unroll
                for (int tx = 0; tx < 2 * HW; ++tx) {
                    const int bx = bx0 + tx;
                    if (bx < 0 || bx >= g.Fb[0]) continue;
                    T wx, dwx;
                    rot_w<T, HW>((T)bx - cx, wx, dwx);
                    sum += wz * wy * wx * kb[bx + (long long)g.Fb[0] * (by + (long long)g.Fb[1] * bz)];
                }
            }
        }
        acc += (double)sum;
    }
    dkref[j] = acc;
}

// Per-step motion sensitivities of the rotating body from the per-block slots (fixed block order):
// g_s[n] += dJ/do, g_uG[n] += dJ/du^G, g_th[n] += dJ/dtheta, g_om[n] += dJ/domega.
template <int D>
__global__ void rot_motion_reduce_kernel(const double* __restrict__ mslot, int nsb, int n_first, int nsteps,
                                         double* __restrict__ g_s, double* __restrict__ g_uG, double* __restrict__ g_th,
                                         double* __restrict__ g_om) {
    constexpr int NV = 2 * D + 2;
    const int st = blockIdx.x;
    if (st >= nsteps || threadIdx.x >= NV) return;
    const int q = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < nsb; ++b) s += mslot[((long long)st * nsb + b) * NV + q];
    const int n = n_first + st;
    if (q < D)
        g_s[n * D + q] += s;
    else if (q < 2 * D)
        g_uG[n * D + q - D] += s;
    else if (q == 2 * D)
        g_th[n] += s;
    else
        g_om[n] += s;
}

}  // namespace lks
