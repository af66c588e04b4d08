// D2Q9 forward and adjoint step kernels in warp-column form.
//
// Each warp owns 32 consecutive x positions (lanes; the 28 lanes 2..29 produce output, the outer two on
// each side only supply x-neighbours) and marches along y over a run of R output rows.  Values at x +- 1
// come from warp shuffles, values at y +- 1 from a rolling window of rows held in registers, so the stencil
// needs no shared memory and no block barrier.  D2Q9 weights factor as w(c) = W(c_x) W(c_y) with
// W(0) = 2/3, W(+-1) = 1/6, which the row-by-row accumulation below uses.
//
// Forward (Sec. 2.2): moment row m is built from raw rows m-1, m, m+1; it pushes
// f_i = w_i [sigma + 3 c.u + c T c] into output rows m + c_y (lanes x + c_x); output row m-1 is complete
// once moment row m has been pushed.  Adjoint: source row r (lambda_n) pushes F-bar into the moments of
// rows r - c_y (lanes x - c_x); moment row r-1 is then complete, and lambda_{n-1} of row r-2 follows from
// the moments of rows r-3..r-1.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"

namespace lks {

constexpr int kLanesOut = 28;  // output columns per warp

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// ------------------------------------------------------------------------------------------------
// Forward step n-1 -> n.
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int R, int WY>
__global__ void __launch_bounds__(32 * WY) fwd2d_kernel(Geom g, FwdArgs<T> a) {
    __shared__ double red[2 * WY];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * kLanesOut;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xo = x0 + lane - 2;                 // this lane's column
    const int xl = wrap(xo, nx);                  // ... wrapped for loads
    const bool lane_out = lane >= 2 && lane < 30 && xo < nx;
    const T A = (T)g.A;
    const T W0 = (T)(2.0 / 3.0), W1 = (T)(1.0 / 6.0), third = (T)(1.0 / 3.0);
    const T* __restrict__ inP = a.in;
    const T* __restrict__ inX = a.in + g.N;
    const T* __restrict__ inY = a.in + 2 * g.N;
    const Pose& P = *a.pose;
    pdl_wait_then_release();

    // load phase: every row this warp reads, issued back to back (memory-level parallelism)
    T pr[R + 4], xr[R + 4], yr[R + 4];
    {
        int yw = wrap(y0 - 2, ny);
#pragma unroll
        for (int it = 0; it < R + 4; ++it) {
            const int gi = yw * nx + xl;
            pr[it] = inP[gi];
            xr[it] = inX[gi];
            yr[it] = inY[gi];
            yw = (yw + 1 == ny) ? 0 : yw + 1;
        }
    }
    // mapping of the output rows (kappa, C from the design grid) while the loads are in flight
    T kap[R], Cm[R], kinv[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        kap[i] = 0;
        Cm[i] = 0;
        kinv[i] = 1;
        const int o = y0 + i;
        int b[2];
        b[0] = box_coord(xo, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        b[1] = box_coord(o, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        if (lane_out && o < ny && b[0] >= 0 && b[1] >= 0) {
            map_node<T, 2, HW, false>(g, P, a.kref, b, kap[i], Cm[i], nullptr, nullptr);
            kinv[i] = (T)1 / ((T)1 + kap[i]);
        }
    }
    // raw window (rows r-2, r-1, r) and output accumulators (rows m-1, m, m+1)
    T p0 = 0, p1 = 0, p2 = 0, ux0 = 0, ux1 = 0, ux2 = 0, uy0 = 0, uy1 = 0, uy2 = 0;
    T aP0 = 0, aP1 = 0, aP2 = 0, aX0 = 0, aX1 = 0, aX2 = 0, aY0 = 0, aY1 = 0, aY2 = 0;
    T jacc = 0, qacc = 0;
    bool unstable = false;
#pragma unroll
    for (int it = 0; it < R + 4; ++it) {
        const int r = y0 - 2 + it;
        p0 = p1; p1 = p2; p2 = pr[it];
        ux0 = ux1; ux1 = ux2; ux2 = xr[it];
        uy0 = uy1; uy1 = uy2; uy2 = yr[it];
        if (it < 2) continue;
        // moment row m = r - 1 from raw rows r-2 (0), r-1 (1), r (2)
        const T uxE = shfl_dn1(ux1), uxW = shfl_up1(ux1), uyE = shfl_dn1(uy1), uyW = shfl_up1(uy1);
        const T sig = (T)3 * p1 - (T)1.5 * (ux1 * ux1 + uy1 * uy1);
        const T Txx = (T)4.5 * ux1 * ux1 + A * (uxE - uxW);
        const T Tyy = (T)4.5 * uy1 * uy1 + A * (uy2 - uy0);
        const T Txy = (T)4.5 * ux1 * uy1 + (T)0.5 * A * ((uyE - uyW) + (ux2 - ux0));
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            const T base = sig + (T)(3 * cy) * uy1 + (T)(cy * cy) * Tyy;
            const T gR = base + (T)3 * ux1 + Txx + (T)(2 * cy) * Txy;  // c = (+1, cy), goes to lane + 1
            const T gL = base - (T)3 * ux1 + Txx - (T)(2 * cy) * Txy;  // c = (-1, cy), goes to lane - 1
            const T fromW = shfl_up1(gR);                               // lane - 1's (+1, cy) value
            const T fromE = shfl_dn1(gL);                               // lane + 1's (-1, cy) value
            const T Wy = cy == 0 ? W0 : W1;
            const T S = Wy * (W1 * (fromW + fromE) + W0 * base);
            const T X = Wy * W1 * (fromW - fromE);
            // output row m + cy
            if (cy == -1) { aP0 += third * S; aX0 += X; aY0 -= S; }
            if (cy == 0) { aP1 += third * S; aX1 += X; }
            if (cy == 1) { aP2 += third * S; aX2 += X; aY2 += S; }
        }
        // output row o = m - 1 = r - 2 is complete
        const int o = r - 2;
        if (it >= 4 && lane_out && o < ny) {
            int xg[2] = {xo, o};
            const T k = kap[it - 4], C = Cm[it - 4];
            const T inv = kinv[it - 4];
            T un0 = (aX0 + k * (pose_uG<T>(P, 0) * C)) * inv;
            T un1 = (aY0 + k * (pose_uG<T>(P, 1) * C)) * inv;
            T uw[2];
            const bool wall = wall_node<T, 2>(g, xg, uw);
            if (wall) {
                un0 = uw[0];
                un1 = uw[1];
            }
            const long long go = (long long)o * nx + xo;
            a.out_p[go] = aP0;
            a.out_u[go] = un0;
            a.out_u[g.N + go] = un1;
            if (!wall) {
                if (a.u_crit2 > (T)0 && !(un0 * un0 + un1 * un1 <= a.u_crit2)) unstable = true;
                if (in_probe<2>(g, xg)) {
                    const T nu = a.dir[0] * un0 + a.dir[1] * un1;
                    jacc += nu;
                    qacc += nu * nu;
                }
            }
        }
        aP0 = aP1; aP1 = aP2; aP2 = 0;
        aX0 = aX1; aX1 = aX2; aX2 = 0;
        aY0 = aY1; aY1 = aY2; aY2 = 0;
    }
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int bx = (int)blockIdx.x - a.jb_lo[0], by = (int)blockIdx.y - a.jb_lo[1];
        if (bx >= 0 && bx < a.jb_n[0] && by >= 0 && by < a.jb_n[1]) {
            store_probe_partials<32 * WY, T>(jacc, qacc, a.jslot, a.jsq, bx + a.jb_n[0] * by, red);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1} with the local shape and motion sensitivities (same algebra as
// adj_step_kernel, in warp-column form).
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int R, int WY>
__global__ void __launch_bounds__(32 * WY) adj2d_kernel(Geom g, AdjArgs<T> a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * kLanesOut;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xo = x0 + lane - 2;
    const int xl = wrap(xo, nx);
    const bool lane_out = lane >= 2 && lane < 30 && xo < nx;
    const T A = (T)g.A;
    const T W0 = (T)(2.0 / 3.0), W1 = (T)(1.0 / 6.0), third = (T)(1.0 / 3.0);
    const T* __restrict__ lP = a.lam_in;
    const T* __restrict__ lX = a.lam_in + g.N;
    const T* __restrict__ lY = a.lam_in + 2 * g.N;
    const Pose& P = *a.pose;
    const long long N = g.N;
    pdl_wait_then_release();

    // load phase: lambda_n of every source row, u_{n-1} of every output row
    T lpr[R + 4], lxr[R + 4], lyr[R + 4], u0r[R], u1r[R];
    {
        int yw = wrap(y0 - 2, ny);
#pragma unroll
        for (int it = 0; it < R + 4; ++it) {
            const int gi = yw * nx + xl;
            lpr[it] = lP[gi];
            lxr[it] = lX[gi];
            lyr[it] = lY[gi];
            yw = (yw + 1 == ny) ? 0 : yw + 1;
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int z = y0 + i;
            const int go = (lane_out && z < ny) ? z * nx + xo : 0;
            u0r[i] = a.u_prev[go];
            u1r[i] = a.u_prev[N + go];
        }
    }
    // Brinkman / wall adjoint factor of every source node: u-bar* = lam_u / (1 + kappa), 0 on walls
    T fac[R + 4];
    {
        int yw = wrap(y0 - 2, ny);
#pragma unroll
        for (int it = 0; it < R + 4; ++it) {
            int xs[2] = {xl, yw};
            T uw[2];
            fac[it] = 1;
            if (wall_node<T, 2>(g, xs, uw)) {
                fac[it] = 0;
            } else {
                int b[2];
                b[0] = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
                b[1] = box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
                if (b[0] >= 0 && b[1] >= 0) fac[it] = adj_inv<T, 2, HW>(g, P, a.kref, a.fac, b);
            }
            yw = (yw + 1 == ny) ? 0 : yw + 1;
        }
    }
    // lambda_u window (rows r-2, r-1, r) for the footprint terms of the output row
    T lx0 = 0, lx1 = 0, lx2 = 0, ly0 = 0, ly1 = 0, ly2 = 0;
    // moment accumulators of rows r+1 (index 2), r (1), r-1 (0); completed rows r-2 (c) and r-3 (p)
    T m0_0 = 0, m0_1 = 0, m0_2 = 0, mx_0 = 0, mx_1 = 0, mx_2 = 0, my_0 = 0, my_1 = 0, my_2 = 0;
    T xx_0 = 0, xx_1 = 0, xx_2 = 0, xy_0 = 0, xy_1 = 0, xy_2 = 0, yy_0 = 0, yy_1 = 0, yy_2 = 0;
    T m0_c = 0, mx_c = 0, my_c = 0, xx_c = 0, xy_c = 0, yy_c = 0;  // row r-2
    T xy_p = 0, yy_p = 0;                                          // row r-3
#pragma unroll
    for (int it = 0; it < R + 4; ++it) {
        const int r = y0 - 2 + it;
        const T lp = lpr[it];
        lx0 = lx1; lx1 = lx2; lx2 = lxr[it];
        ly0 = ly1; ly1 = ly2; ly2 = lyr[it];
        // p-bar* = lam_p, u-bar* = lam_u / (1 + kappa) (0 on walls)
        const T ubx = lx2 * fac[it], uby = ly2 * fac[it];
        // push F-bar of source row r into the moments of rows r - cy
        const T pW = shfl_up1(lp), pE = shfl_dn1(lp);
        const T xW = shfl_up1(ubx), xE = shfl_dn1(ubx);
        const T yW = shfl_up1(uby), yE = shfl_dn1(uby);
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            const T FL = third * pW - xW + (T)cy * yW;   // source x-1: c = (-1, cy)
            const T FC = third * lp + (T)cy * uby;       // source x:   c = (0, cy)
            const T FR = third * pE + xE + (T)cy * yE;   // source x+1: c = (+1, cy)
            const T Wy = cy == 0 ? W0 : W1;
            const T S = Wy * (W1 * (FL + FR) + W0 * FC);
            const T Dd = Wy * W1 * (FR - FL);
            const T Sx = Wy * W1 * (FL + FR);
            // moment row y = r - cy
            if (cy == 1) {  // row r-1
                m0_0 += S; mx_0 += Dd; my_0 += S; xx_0 += Sx; xy_0 += Dd; yy_0 += S;
            } else if (cy == 0) {  // row r
                m0_1 += S; mx_1 += Dd; xx_1 += Sx;
            } else {  // row r+1
                m0_2 += S; mx_2 += Dd; my_2 -= S; xx_2 += Sx; xy_2 -= Dd; yy_2 += S;
            }
        }
        // moment row r-1 is complete: it becomes the "next" row of the output row r-2
        if (it >= 4) {
            const int z = r - 2;
            // lambda_{n-1} at row z from moments of rows z-1 (p), z (c), z+1 (0)
            const T xxE = shfl_dn1(xx_c), xxW = shfl_up1(xx_c), xyE = shfl_dn1(xy_c), xyW = shfl_up1(xy_c);
            if (lane_out && z < ny) {
                const long long go = (long long)z * nx + xo;
                const T u0 = u0r[it - 4], u1 = u1r[it - 4];
                T vx = (T)3 * mx_c - (T)3 * u0 * m0_c + (T)9 * (xx_c * u0 + xy_c * u1) + A * ((xxW - xxE) + (xy_p - xy_0));
                T vy = (T)3 * my_c - (T)3 * u1 * m0_c + (T)9 * (xy_c * u0 + yy_c * u1) + A * ((xyW - xyE) + (yy_p - yy_0));
                int xg[2] = {xo, z};
                T uw[2];
                const bool wall = wall_node<T, 2>(g, xg, uw);
                if (a.src && !wall && in_probe<2>(g, xg)) {
                    const T f = src_factor(a, a.dir[0] * u0 + a.dir[1] * u1);
                    vx += a.phi_dir[0] * f;
                    vy += a.phi_dir[1] * f;
                }
                a.lam_out[go] = (T)3 * m0_c;
                a.lam_out[N + go] = vx;
                a.lam_out[2 * N + go] = vy;
                // record lam_u and u_n on the footprint box for the segment's sensitivity pass
                const int b0 = box_coord(xo, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
                const int b1 = box_coord(z, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
                if (b0 >= 0 && b1 >= 0) {
                    const long long bl = b0 + (long long)g.Fb[0] * b1;
                    a.boxbuf[bl] = wall ? (T)0 : lx0;
                    a.boxbuf[g.Fbn + bl] = wall ? (T)0 : ly0;
                    a.boxbuf[2 * g.Fbn + bl] = a.u_cur[go];
                    a.boxbuf[3 * g.Fbn + bl] = a.u_cur[N + go];
                }
            }
        }
        // roll: completed row r-1 becomes the output row of the next iteration
        xy_p = xy_c; yy_p = yy_c;
        m0_c = m0_0; mx_c = mx_0; my_c = my_0; xx_c = xx_0; xy_c = xy_0; yy_c = yy_0;
        m0_0 = m0_1; mx_0 = mx_1; my_0 = my_1; xx_0 = xx_1; xy_0 = xy_1; yy_0 = yy_1;
        m0_1 = m0_2; mx_1 = mx_2; my_1 = my_2; xx_1 = xx_2; xy_1 = xy_2; yy_1 = yy_2;
        m0_2 = 0; mx_2 = 0; my_2 = 0; xx_2 = 0; xy_2 = 0; yy_2 = 0;
    }
}

}  // namespace lks
