// D2Q9 forward and adjoint step kernels in vectorised warp-column form, for large grids.
//
// Each lane owns two adjacent columns (x = x0 - 2 + 2 lane and x + 1) and moves them with one 8- or 16-byte load
// or store per field; a warp covers 64 columns of which the 60 in lanes 1..30 are output.  A column's
// x-neighbours are either its partner in the same lane or a column of the adjacent lane (one warp shuffle per
// field and direction, half as many as with one column per lane).  The warp marches along y over R rows with a
// rolling window of three rows in registers and a prefetch of two rows ahead; per-lane and per-row tests (walls,
// probe box, footprint box) are hoisted out of the node work.  The grid's x extent must be even (pairs of columns
// never straddle the periodic seam).  The arithmetic per node is that of fwd_step_kernel / adj_step_kernel.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"

namespace lks {

constexpr int kVecCols = 60;  // output columns per warp

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ T shfl_u(T v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shfl_d(T v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// Wall side of a coordinate on a non-periodic axis (-1: none, 0: plane 0, 1: plane n-1).
__device__ __forceinline__ int wall_side(int x, int n, int periodic) {
    return periodic ? -1 : (x == 0 ? 0 : (x == n - 1 ? 1 : -1));
}

// ------------------------------------------------------------------------------------------------
// Forward step n-1 -> n.
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int R>
__global__ void __launch_bounds__(128) fwd2v_kernel(Geom g, FwdArgs<T> a) {
    using V = typename Vec2<T>::type;
    constexpr int WY = 4;
    __shared__ double red[WY];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * kVecCols;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xe = x0 - 2 + 2 * lane;     // even column of this lane (odd column xe + 1)
    const int xl = wrap(xe, nx);          // even too, as nx is even
    const bool lane_out = lane >= 1 && lane <= 30 && xe < nx;
    const T A = (T)g.A;
    const T W0 = (T)(2.0 / 3.0), W1 = (T)(1.0 / 6.0), third = (T)(1.0 / 3.0);
    const V* __restrict__ inP = reinterpret_cast<const V*>(a.in);
    const V* __restrict__ inX = reinterpret_cast<const V*>(a.in + g.N);
    const V* __restrict__ inY = reinterpret_cast<const V*>(a.in + 2 * g.N);
    const Pose& P = *a.pose;
    // per-lane invariants
    const int bxe = box_coord(xe, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int bxo = box_coord(xe + 1, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int wxe = wall_side(xe, nx, g.periodic[0]), wxo = wall_side(xe + 1, nx, g.periodic[0]);
    const bool pxe = xe >= g.probe_lo[0] && xe < g.probe_hi[0];
    const bool pxo = xe + 1 >= g.probe_lo[0] && xe + 1 < g.probe_hi[0];
    const int half = nx >> 1;
    pdl_wait_then_release();

    auto load = [&](int r, V& p, V& ux, V& uy) {
        const int gi = wrap(r, ny) * half + (xl >> 1);
        p = inP[gi];
        ux = inX[gi];
        uy = inY[gi];
    };
    // rolling window (rows r-2, r-1, r) and prefetch (rows r+1, r+2)
    V p0, x0v, y0v, p1, x1v, y1v, p2, x2v, y2v, pA, xA, yA, pB, xB, yB;
    load(y0 - 2, p0, x0v, y0v);
    load(y0 - 1, p1, x1v, y1v);
    load(y0, pA, xA, yA);
    load(y0 + 1, pB, xB, yB);
    // output accumulators of rows m-1 (0), m (1), m+1 (2); e = even column, o = odd column
    T aP0e = 0, aP0o = 0, aX0e = 0, aX0o = 0, aY0e = 0, aY0o = 0;
    T aP1e = 0, aP1o = 0, aX1e = 0, aX1o = 0, aY1e = 0, aY1o = 0;
    T aP2e = 0, aP2o = 0, aX2e = 0, aX2o = 0, aY2e = 0, aY2o = 0;
    T jacc = 0;
    bool unstable = false;

#pragma unroll 1
    for (int r = y0; r <= y0 + R + 1; ++r) {
        p2 = pA; x2v = xA; y2v = yA;
        pA = pB; xA = xB; yA = yB;
        if (r + 2 <= y0 + R + 1) load(r + 2, pB, xB, yB);
        // moment row m = r - 1 from rows r-2 (0), r-1 (1), r (2)
        const T uxe = x1v.x, uxo = x1v.y, uye = y1v.x, uyo = y1v.y;
        const T uxW = shfl_u(uxo), uxE = shfl_d(uxe), uyW = shfl_u(uyo), uyE = shfl_d(uye);
        const T sige = (T)3 * p1.x - (T)1.5 * (uxe * uxe + uye * uye);
        const T sigo = (T)3 * p1.y - (T)1.5 * (uxo * uxo + uyo * uyo);
        const T Txxe = (T)4.5 * uxe * uxe + A * (uxo - uxW);
        const T Txxo = (T)4.5 * uxo * uxo + A * (uxE - uxe);
        const T Tyye = (T)4.5 * uye * uye + A * (y2v.x - y0v.x);
        const T Tyyo = (T)4.5 * uyo * uyo + A * (y2v.y - y0v.y);
        const T Txye = (T)4.5 * uxe * uye + (T)0.5 * A * ((uyo - uyW) + (x2v.x - x0v.x));
        const T Txyo = (T)4.5 * uxo * uyo + (T)0.5 * A * ((uyE - uye) + (x2v.y - x0v.y));
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            const T be = sige + (T)(3 * cy) * uye + (T)(cy * cy) * Tyye;
            const T bo = sigo + (T)(3 * cy) * uyo + (T)(cy * cy) * Tyyo;
            const T gRe = be + (T)3 * uxe + Txxe + (T)(2 * cy) * Txye;  // (+1, cy) from the even column
            const T gLe = be - (T)3 * uxe + Txxe - (T)(2 * cy) * Txye;  // (-1, cy)
            const T gRo = bo + (T)3 * uxo + Txxo + (T)(2 * cy) * Txyo;
            const T gLo = bo - (T)3 * uxo + Txxo - (T)(2 * cy) * Txyo;
            const T inWe = shfl_u(gRo);  // into the even column from x - 1 (previous lane's odd column)
            const T inEo = shfl_d(gLe);  // into the odd column from x + 1 (next lane's even column)
            const T Wy = cy == 0 ? W0 : W1;
            const T Se = Wy * (W1 * (inWe + gLo) + W0 * be), Xe = Wy * W1 * (inWe - gLo);
            const T So = Wy * (W1 * (gRe + inEo) + W0 * bo), Xo = Wy * W1 * (gRe - inEo);
            if (cy == -1) { aP0e += third * Se; aX0e += Xe; aY0e -= Se; aP0o += third * So; aX0o += Xo; aY0o -= So; }
            if (cy == 0) { aP1e += third * Se; aX1e += Xe; aP1o += third * So; aX1o += Xo; }
            if (cy == 1) { aP2e += third * Se; aX2e += Xe; aY2e += Se; aP2o += third * So; aX2o += Xo; aY2o += So; }
        }
        // output row o = r - 2
        const int o = r - 2;
        if (o >= y0 && lane_out && o < ny) {
            const int wy = wall_side(o, ny, g.periodic[1]);
            const int by = box_coord(o, P.xs[1], g.Fb[1], ny, g.periodic[1]);
            const bool py = o >= g.probe_lo[1] && o < g.probe_hi[1];
            // Brinkman with the mapped kappa, walls, stability and objective for one column of the pair
            auto finish = [&](T& u0, T& u1, int bx, int wx, bool px) {
                if (bx >= 0 && by >= 0) {
                    const int b[2] = {bx, by};
                    T kap, C;
                    map_node<T, 2, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
                    const T inv = (T)1 / ((T)1 + kap);
                    u0 = (u0 + kap * (pose_uG<T>(P, 0) * C)) * inv;
                    u1 = (u1 + kap * (pose_uG<T>(P, 1) * C)) * inv;
                }
                if (wx >= 0 || wy >= 0) {
                    // later axes win where wall planes meet
                    const int ax = wy >= 0 ? 1 : 0, side = wy >= 0 ? wy : wx;
                    u0 = (T)g.wall_u[ax][side][0];
                    u1 = (T)g.wall_u[ax][side][1];
                } else {
                    if (a.u_crit2 > (T)0 && !(u0 * u0 + u1 * u1 <= a.u_crit2)) unstable = true;
                    if (py && px) jacc += a.dir[0] * u0 + a.dir[1] * u1;
                }
            };
            T ue0 = aX0e, ue1 = aY0e, uo0 = aX0o, uo1 = aY0o;
            finish(ue0, ue1, bxe, wxe, pxe);
            finish(uo0, uo1, bxo, wxo, pxo);
            const int go = o * half + (xe >> 1);
            V* outP = reinterpret_cast<V*>(a.out_p);
            V* outX = reinterpret_cast<V*>(a.out_u);
            V* outY = reinterpret_cast<V*>(a.out_u + g.N);
            V vp, vx, vy;
            vp.x = aP0e; vp.y = aP0o;
            vx.x = ue0; vx.y = uo0;
            vy.x = ue1; vy.y = uo1;
            outP[go] = vp;
            outX[go] = vx;
            outY[go] = vy;
        }
        p0 = p1; x0v = x1v; y0v = y1v;
        p1 = p2; x1v = x2v; y1v = y2v;
        aP0e = aP1e; aP0o = aP1o; aX0e = aX1e; aX0o = aX1o; aY0e = aY1e; aY0o = aY1o;
        aP1e = aP2e; aP1o = aP2o; aX1e = aX2e; aX1o = aX2o; aY1e = aY2e; aY1o = aY2o;
        aP2e = 0; aP2o = 0; aX2e = 0; aX2o = 0; aY2e = 0; aY2o = 0;
    }
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int bx = (int)blockIdx.x - a.jb_lo[0], by = (int)blockIdx.y - a.jb_lo[1];
        if (bx >= 0 && bx < a.jb_n[0] && by >= 0 && by < a.jb_n[1]) {
            T v[1] = {jacc};
            double s[1];
            block_sum<32 * WY, 1, T>(v, s, red);
            if (threadIdx.x == 0) a.jslot[bx + a.jb_n[0] * by] = s[0];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1}, recording lam_u and u_n on the footprint box.
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int R>
__global__ void __launch_bounds__(128, 5) adj2v_kernel(Geom g, AdjArgs<T> a) {
    using V = typename Vec2<T>::type;
    constexpr int WY = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = g.n[0], ny = g.n[1];
    const long long N = g.N;
    const int x0 = blockIdx.x * kVecCols;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xe = x0 - 2 + 2 * lane;
    const int xl = wrap(xe, nx);
    const bool lane_out = lane >= 1 && lane <= 30 && xe < nx;
    const T A = (T)g.A;
    const T W0 = (T)(2.0 / 3.0), W1 = (T)(1.0 / 6.0), third = (T)(1.0 / 3.0);
    const V* __restrict__ lP = reinterpret_cast<const V*>(a.lam_in);
    const V* __restrict__ lX = reinterpret_cast<const V*>(a.lam_in + N);
    const V* __restrict__ lY = reinterpret_cast<const V*>(a.lam_in + 2 * N);
    const V* __restrict__ upX = reinterpret_cast<const V*>(a.u_prev);
    const V* __restrict__ upY = reinterpret_cast<const V*>(a.u_prev + N);
    const Pose& P = *a.pose;
    const int half = nx >> 1;
    // per-lane invariants: source columns (wrapped) and output columns
    const int sbxe = box_coord(xl, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int sbxo = box_coord(xl + 1, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int swxe = wall_side(xl, nx, g.periodic[0]), swxo = wall_side(xl + 1, nx, g.periodic[0]);
    const int bxe = box_coord(xe, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int bxo = box_coord(xe + 1, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const bool pxe = xe >= g.probe_lo[0] && xe < g.probe_hi[0];
    const bool pxo = xe + 1 >= g.probe_lo[0] && xe + 1 < g.probe_hi[0];
    pdl_wait_then_release();

    auto load = [&](int r, V& p, V& ux, V& uy) {
        const int gi = wrap(r, ny) * half + (xl >> 1);
        p = lP[gi];
        ux = lX[gi];
        uy = lY[gi];
    };
    // Brinkman / wall adjoint factor of a source node: 1/(1 + kappa) off the walls, 0 on them
    auto factor = [&](int yw, int bx, int wx) -> T {
        if (wx >= 0 || wall_side(yw, ny, g.periodic[1]) >= 0) return (T)0;
        const int by = box_coord(yw, P.xs[1], g.Fb[1], ny, g.periodic[1]);
        if (bx < 0 || by < 0) return (T)1;
        const int b[2] = {bx, by};
        return adj_inv<T, 2, HW>(g, P, a.kref, a.fac, b);
    };
    V pA, xA, yA, pB, xB, yB;
    load(y0 - 2, pA, xA, yA);
    load(y0 - 1, pB, xB, yB);
    // u_{n-1} of the output rows, two rows ahead (row z is consumed at iteration r = z + 2)
    auto load_u = [&](int z, V& u0, V& u1) {
        const int gz = (lane_out && z < ny) ? z * half + (xe >> 1) : 0;
        u0 = upX[gz];
        u1 = upY[gz];
    };
    V uxA, uyA, uxB, uyB;
    load_u(y0, uxA, uyA);
    load_u(y0 + 1, uxB, uyB);
    // moment accumulators of rows r+1 (2), r (1), r-1 (0); completed rows r-2 (c), r-3 (p); e/o columns
    T m0e0 = 0, m0o0 = 0, mxe0 = 0, mxo0 = 0, mye0 = 0, myo0 = 0, xxe0 = 0, xxo0 = 0, xye0 = 0, xyo0 = 0, yye0 = 0, yyo0 = 0;
    T m0e1 = 0, m0o1 = 0, mxe1 = 0, mxo1 = 0, mye1 = 0, myo1 = 0, xxe1 = 0, xxo1 = 0, xye1 = 0, xyo1 = 0, yye1 = 0, yyo1 = 0;
    T m0e2 = 0, m0o2 = 0, mxe2 = 0, mxo2 = 0, mye2 = 0, myo2 = 0, xxe2 = 0, xxo2 = 0, xye2 = 0, xyo2 = 0, yye2 = 0, yyo2 = 0;
    T m0ec = 0, m0oc = 0, mxec = 0, mxoc = 0, myec = 0, myoc = 0, xxec = 0, xxoc = 0, xyec = 0, xyoc = 0, yyec = 0, yyoc = 0;
    T xyep = 0, xyop = 0, yyep = 0, yyop = 0;

#pragma unroll 1
    for (int r = y0 - 2; r <= y0 + R + 1; ++r) {
        const V lp = pA, lxv = xA, lyv = yA;
        pA = pB; xA = xB; yA = yB;
        if (r + 2 <= y0 + R + 1) load(r + 2, pB, xB, yB);
        // source row r: p-bar* = lam_p, u-bar* = lam_u * factor
        const int yw = wrap(r, ny);
        const T fe = factor(yw, sbxe, swxe), fo = factor(yw, sbxo, swxo);
        const T pe = lp.x, po = lp.y, ue = lxv.x * fe, uo = lxv.y * fo, ve = lyv.x * fe, vo = lyv.y * fo;
        // neighbours: x-1 of the even column is the previous lane's odd column, x+1 of the odd column the next
        // lane's even column
        const T pW = shfl_u(po), uW = shfl_u(uo), vW = shfl_u(vo);
        const T pE = shfl_d(pe), uE = shfl_d(ue), vE = shfl_d(ve);
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            // even column: sources x-1 (W), x (e), x+1 (o)
            const T FLe = third * pW - uW + (T)cy * vW;
            const T FCe = third * pe + (T)cy * ve;
            const T FRe = third * po + uo + (T)cy * vo;
            // odd column: sources x-1 (e), x (o), x+1 (E)
            const T FLo = third * pe - ue + (T)cy * ve;
            const T FCo = third * po + (T)cy * vo;
            const T FRo = third * pE + uE + (T)cy * vE;
            const T Wy = cy == 0 ? W0 : W1;
            const T Se = Wy * (W1 * (FLe + FRe) + W0 * FCe), De = Wy * W1 * (FRe - FLe), Sxe = Wy * W1 * (FLe + FRe);
            const T So = Wy * (W1 * (FLo + FRo) + W0 * FCo), Do = Wy * W1 * (FRo - FLo), Sxo = Wy * W1 * (FLo + FRo);
            if (cy == 1) {  // moment row r-1
                m0e0 += Se; mxe0 += De; mye0 += Se; xxe0 += Sxe; xye0 += De; yye0 += Se;
                m0o0 += So; mxo0 += Do; myo0 += So; xxo0 += Sxo; xyo0 += Do; yyo0 += So;
            } else if (cy == 0) {  // row r
                m0e1 += Se; mxe1 += De; xxe1 += Sxe;
                m0o1 += So; mxo1 += Do; xxo1 += Sxo;
            } else {  // row r+1
                m0e2 += Se; mxe2 += De; mye2 -= Se; xxe2 += Sxe; xye2 -= De; yye2 += Se;
                m0o2 += So; mxo2 += Do; myo2 -= So; xxo2 += Sxo; xyo2 -= Do; yyo2 += So;
            }
        }
        // lambda_{n-1} of row z = r - 2 from moment rows z-1 (p), z (c), z+1 (0)
        const int z = r - 2;
        if (z >= y0) {
            const V u0 = uxA, u1 = uyA;
            uxA = uxB;
            uyA = uyB;
            if (z + 2 <= y0 + R - 1) load_u(z + 2, uxB, uyB);
            const T xxW = shfl_u(xxoc), xxE = shfl_d(xxec), xyW = shfl_u(xyoc), xyE = shfl_d(xyec);
            if (lane_out && z < ny) {
                const int go = z * half + (xe >> 1);
                T vxe = (T)3 * mxec - (T)3 * u0.x * m0ec + (T)9 * (xxec * u0.x + xyec * u1.x) +
                        A * ((xxW - xxoc) + (xyep - xye0));
                T vye = (T)3 * myec - (T)3 * u1.x * m0ec + (T)9 * (xyec * u0.x + yyec * u1.x) +
                        A * ((xyW - xyoc) + (yyep - yye0));
                T vxo = (T)3 * mxoc - (T)3 * u0.y * m0oc + (T)9 * (xxoc * u0.y + xyoc * u1.y) +
                        A * ((xxec - xxE) + (xyop - xyo0));
                T vyo = (T)3 * myoc - (T)3 * u1.y * m0oc + (T)9 * (xyoc * u0.y + yyoc * u1.y) +
                        A * ((xyec - xyE) + (yyop - yyo0));
                const int wy = wall_side(z, ny, g.periodic[1]);
                const bool we = wy >= 0 || wall_side(xe, nx, g.periodic[0]) >= 0;
                const bool wo = wy >= 0 || wall_side(xe + 1, nx, g.periodic[0]) >= 0;
                const bool py = a.src && z >= g.probe_lo[1] && z < g.probe_hi[1];
                if (py && pxe && !we) {
                    vxe += a.phi_dir[0];
                    vye += a.phi_dir[1];
                }
                if (py && pxo && !wo) {
                    vxo += a.phi_dir[0];
                    vyo += a.phi_dir[1];
                }
                V* oP = reinterpret_cast<V*>(a.lam_out);
                V* oX = reinterpret_cast<V*>(a.lam_out + N);
                V* oY = reinterpret_cast<V*>(a.lam_out + 2 * N);
                V t;
                t.x = (T)3 * m0ec; t.y = (T)3 * m0oc;
                oP[go] = t;
                t.x = vxe; t.y = vxo;
                oX[go] = t;
                t.x = vye; t.y = vyo;
                oY[go] = t;
                const int by = box_coord(z, P.xs[1], g.Fb[1], ny, g.periodic[1]);
                if (by >= 0) {
                    for (int s = 0; s < 2; ++s) {
                        const int bx = s == 0 ? bxe : bxo;
                        if (bx < 0) continue;
                        const bool w = s == 0 ? we : wo;
                        const long long bl = bx + (long long)g.Fb[0] * by;
                        const long long gi = (long long)z * nx + xe + s;
                        a.boxbuf[bl] = w ? (T)0 : a.lam_in[N + gi];
                        a.boxbuf[g.Fbn + bl] = w ? (T)0 : a.lam_in[2 * N + gi];
                        a.boxbuf[2 * g.Fbn + bl] = a.u_cur[gi];
                        a.boxbuf[3 * g.Fbn + bl] = a.u_cur[N + gi];
                    }
                }
            }
        }
        // roll the moment rows
        xyep = xyec; xyop = xyoc; yyep = yyec; yyop = yyoc;
        m0ec = m0e0; m0oc = m0o0; mxec = mxe0; mxoc = mxo0; myec = mye0; myoc = myo0;
        xxec = xxe0; xxoc = xxo0; xyec = xye0; xyoc = xyo0; yyec = yye0; yyoc = yyo0;
        m0e0 = m0e1; m0o0 = m0o1; mxe0 = mxe1; mxo0 = mxo1; mye0 = mye1; myo0 = myo1;
        xxe0 = xxe1; xxo0 = xxo1; xye0 = xye1; xyo0 = xyo1; yye0 = yye1; yyo0 = yyo1;
        m0e1 = m0e2; m0o1 = m0o2; mxe1 = mxe2; mxo1 = mxo2; mye1 = mye2; myo1 = myo2;
        xxe1 = xxe2; xxo1 = xxo2; xye1 = xye2; xyo1 = xyo2; yye1 = yye2; yyo1 = yyo2;
        m0e2 = 0; m0o2 = 0; mxe2 = 0; mxo2 = 0; mye2 = 0; myo2 = 0;
        xxe2 = 0; xxo2 = 0; xye2 = 0; xyo2 = 0; yye2 = 0; yyo2 = 0;
    }
}

}  // namespace lks
