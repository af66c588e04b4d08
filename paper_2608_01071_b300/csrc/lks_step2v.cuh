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

#include <type_traits>

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

// Arithmetic on (even, odd) column pairs: FP32 pairs use the packed FP32x2 instructions (one issue for both
// columns, same rounding as the scalar ones; a - b is fma(b, -1, a)), FP64 pairs are component-wise.
__device__ __forceinline__ float2 vmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 vmk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename T>
__device__ __forceinline__ typename Vec2<T>::type vsplat(double a) {
    return vmk((T)a, (T)a);
}

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

// kappa and C (Eqs. kappa, u_s) at footprint-box node (bx, by) for the FP32 state and the hat kernel: the 2 x 2 taps
// (weight 0 off the design grid), every operation an explicitly rounded intrinsic, so that the forward step and
// box_fac_hat2_kernel give kappa and 1 / (1 + kappa) bit for bit alike whatever the compiler contracts around them.
__device__ __forceinline__ void map_hat2(const Geom& g, const Pose& P, const float* __restrict__ kref, int bx, int by,
                                         float& kap, float& C) {
    float wx[2], wy[2], sx = 0.f, sy = 0.f;
    int ix[2], iy[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int jx = bx - 1 + k, jy = by - 1 + k;
        const bool vx = jx >= 0 && jx < g.nde[0], vy = jy >= 0 && jy < g.nde[1];
        wx[k] = vx ? P.wf[0][k] : 0.f;
        wy[k] = vy ? P.wf[1][k] : 0.f;
        ix[k] = vx ? jx : 0;
        iy[k] = vy ? jy : 0;
        sx = __fadd_rn(sx, wx[k]);
        sy = __fadd_rn(sy, wy[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx)
            s = __fmaf_rn(__fmul_rn(wx[kx], wy[ky]), kref[ix[kx] + g.nde[0] * iy[ky]], s);
    kap = s;
    C = __fmul_rn(sx, sy);
}

// ------------------------------------------------------------------------------------------------
// Forward step n-1 -> n.
// ------------------------------------------------------------------------------------------------
// With the FP32 state and the hat kernel the Brinkman step maps kappa with map_hat2 and, when a.fac_out is set (the
// recomputation of the reverse sweep), also stores 1 / (1 + kappa) of its footprint-box nodes for the adjoint.
// The input rows arrive by asynchronous copies into a per-warp ring of kFwd2vDepth rows in shared memory,
// kFwd2vDepth - 1 rows ahead of use; each lane copies and reads back only its own column pair, so the ring needs no
// barrier, and many rows are in flight without holding them in registers.
constexpr int kFwd2vDepth = 6;
template <typename T, int HW>
constexpr bool kHat2f = std::is_same<T, float>::value && HW == 1;
template <typename T>
constexpr size_t smem2v_fwd() {
    return sizeof(typename Vec2<T>::type) * 4 * kFwd2vDepth * 3 * 32;
}

template <typename T, int HW, int R>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (HW == 1 ? 7 : 5) : 4) fwd2v_kernel(Geom g, FwdArgs<T> a) {
    using V = typename Vec2<T>::type;
    constexpr int WY = 4, DEPTH = kFwd2vDepth;
    __shared__ double red[2 * WY];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V* ring = reinterpret_cast<V*>(smem_raw) + (size_t)warp * DEPTH * 96;  // [DEPTH][p, u_x, u_y][32]
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * kVecCols;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xe = x0 - 2 + 2 * lane;     // even column of this lane (odd column xe + 1)
    const int xl = wrap(xe, nx);          // even too, as nx is even
    const bool lane_out = lane >= 1 && lane <= 30 && xe < nx;
    const T A = (T)g.A;
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

    // input row t = y0 - 2 + t (t = 0 .. R + 3) into ring slot t mod DEPTH, one copy group per row
    constexpr int NRW = R + 4;
    auto issue = [&](int t) {
        if (t < NRW) {
            V* sv = ring + (t % DEPTH) * 96;
            const int gi = wrap(y0 - 2 + t, ny) * half + (xl >> 1);
            cp_async<sizeof(V)>(sv + lane, inP + gi);
            cp_async<sizeof(V)>(sv + 32 + lane, inX + gi);
            cp_async<sizeof(V)>(sv + 64 + lane, inY + gi);
        }
        cp_async_commit();
    };
    // row t, once it has landed (its slot is refilled DEPTH - 1 rows later)
    auto take = [&](int t, V& p, V& ux, V& uy) {
        issue(t + DEPTH - 1);
        cp_async_wait<DEPTH - 1>();
        const V* sv = ring + (t % DEPTH) * 96;
        p = sv[lane];
        ux = sv[32 + lane];
        uy = sv[64 + lane];
    };
#pragma unroll
    for (int t = 0; t < DEPTH - 1; ++t) issue(t);
    // rolling window of input rows (r-2, r-1, r) and output accumulators of rows m-1, m, m+1 (m = r - 1) as (even,
    // odd) pairs (sum_i f_i, u*_x, u*_y): three sets of each take those roles in turn, the loop body unrolled three
    // times with the roles renamed instead of moving the sets between registers every row
    struct Row { V p, x, y; };
    struct Acc { V P, X, Y; };
    Row Wa, Wb, Wc;
    take(0, Wa.p, Wa.x, Wa.y);
    take(1, Wb.p, Wb.x, Wb.y);
    const V zero = vsplat<T>(0.0);
    Acc Aa{zero, zero, zero}, Ab = Aa, Ac = Aa;
    const V c3 = vsplat<T>(3.0), cm15 = vsplat<T>(-1.5), c45 = vsplat<T>(4.5), vA = vmk(A, A),
            vhA = vmk((T)0.5 * A, (T)0.5 * A);
    bool unstable = false;

    // input row r = y0 + k (loop row k); w0, w1, w2 = rows r-2, r-1, r; a0, a1, a2 = accumulators of rows r-2, r-1, r
    auto step = [&](int k, Row& w0, Row& w1, Row& w2, Acc& a0, Acc& a1, Acc& a2) {
        const int r = y0 + k;
        take(k + 2, w2.p, w2.x, w2.y);
        // moment row m = r - 1 from rows r-2, r-1, r; the x-neighbours of the pair are
        // (x - 1) = (previous lane's odd, even) and (x + 1) = (odd, next lane's even)
        const V ux = w1.x, uy = w1.y;
        const V uxL = vmk(shfl_u(ux.y), ux.x), uxR = vmk(ux.y, shfl_d(ux.x));
        const V uyL = vmk(shfl_u(uy.y), uy.x), uyR = vmk(uy.y, shfl_d(uy.x));
        const V uxx = vmul(ux, ux), uyy = vmul(uy, uy);
        const V sig = vfma(cm15, vadd(uxx, uyy), vmul(c3, w1.p));
        const V Txx = vfma(c45, uxx, vmul(vA, vsub(uxR, uxL)));
        const V Tyy = vfma(c45, uyy, vmul(vA, vsub(w2.y, w0.y)));
        const V Txy = vfma(c45, vmul(ux, uy), vmul(vhA, vadd(vsub(uyR, uyL), vsub(w2.x, w0.x))));
        const V ux3 = vmul(c3, ux);
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            // b = sigma + 3 cy u_y + cy^2 T_yy; g(+-1, cy) = b +- 3 u_x + T_xx +- 2 cy T_xy
            const V b = cy == 0 ? sig : vadd(vfma(vsplat<T>(3.0 * cy), uy, sig), Tyy);
            const V cb = vadd(b, Txx);
            const V gR = cy == 0 ? vadd(cb, ux3) : vfma(vsplat<T>(2.0 * cy), Txy, vadd(cb, ux3));
            const V gL = cy == 0 ? vsub(cb, ux3) : vfma(vsplat<T>(-2.0 * cy), Txy, vsub(cb, ux3));
            // streamed into the pair from x - 1 (gR of the left neighbours) and from x + 1 (gL of the right)
            const V FL = vmk(shfl_u(gR.y), gR.x), FR = vmk(gL.y, shfl_d(gL.x));
            const double Wy = cy == 0 ? 2.0 / 3.0 : 1.0 / 6.0;
            const V S = vfma(vsplat<T>(Wy / 6.0), vadd(FL, FR), vmul(vsplat<T>(Wy * 2.0 / 3.0), b));
            const V X = vmul(vsplat<T>(Wy / 6.0), vsub(FL, FR));
            if (cy == -1) { a0.P = vadd(a0.P, S); a0.X = vadd(a0.X, X); a0.Y = vsub(a0.Y, S); }
            if (cy == 0) { a1.P = vadd(a1.P, S); a1.X = vadd(a1.X, X); }
            if (cy == 1) { a2.P = vadd(a2.P, S); a2.X = vadd(a2.X, X); a2.Y = vadd(a2.Y, S); }
        }
        // output row o = r - 2
        const int o = r - 2;
        if (o >= y0 && lane_out && o < ny) {
            const int wy = wall_side(o, ny, g.periodic[1]);
            const int by = box_coord(o, P.xs[1], g.Fb[1], ny, g.periodic[1]);
            // Brinkman with the mapped kappa, walls and stability for one column of the pair
            auto finish = [&](T& u0, T& u1, int bx, int wx) {
                if (bx >= 0 && by >= 0) {
                    T kap, C, inv;
                    if constexpr (kHat2f<T, HW>) {
                        map_hat2(g, P, a.kref, bx, by, kap, C);
                        inv = __fdiv_rn(1.f, __fadd_rn(1.f, kap));
                        if (a.fac_out != nullptr) a.fac_out[bx + g.Fb[0] * by] = inv;
                    } else {
                        const int b[2] = {bx, by};
                        map_node<T, 2, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
                        inv = (T)1 / ((T)1 + kap);
                    }
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
                }
            };
            T ue0 = a0.X.x, ue1 = a0.Y.x, uo0 = a0.X.y, uo1 = a0.Y.y;
            finish(ue0, ue1, bxe, wxe);
            finish(uo0, uo1, bxo, wxo);
            const int go = o * half + (xe >> 1);
            V* outP = reinterpret_cast<V*>(a.out_p);
            V* outX = reinterpret_cast<V*>(a.out_u);
            V* outY = reinterpret_cast<V*>(a.out_u + g.N);
            V vp, vx, vy;
            vp = vmul(vsplat<T>(1.0 / 3.0), a0.P);
            vx.x = ue0; vx.y = uo0;
            vy.x = ue1; vy.y = uo1;
            outP[go] = vp;
            outX[go] = vx;
            outY[go] = vy;
        }
        a0 = Acc{zero, zero, zero};  // the output row's set starts row r+1
    };
    constexpr int NIT = R + 2;  // rows r = y0 .. y0 + R + 1
    int k = 0;
#pragma unroll 1
    for (; k + 3 <= NIT; k += 3) {
        step(k, Wa, Wb, Wc, Aa, Ab, Ac);
        step(k + 1, Wb, Wc, Wa, Ab, Ac, Aa);
        step(k + 2, Wc, Wa, Wb, Ac, Aa, Ab);
    }
    if (NIT % 3 >= 1) step(k, Wa, Wb, Wc, Aa, Ab, Ac);
    if (NIT % 3 >= 2) step(k + 1, Wb, Wc, Wa, Ab, Ac, Aa);
    cp_async_wait<0>();
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int bx = (int)blockIdx.x - a.jb_lo[0], by = (int)blockIdx.y - a.jb_lo[1];
        if (bx >= 0 && bx < a.jb_n[0] && by >= 0 && by < a.jb_n[1]) {
            // objective partials from this thread's own outputs, re-read after the march so that the march
            // keeps no accumulators (same nodes and order: rows up, even column before odd)
            T jacc = 0, qacc = 0;
            if (lane_out) {
                const V* oX = reinterpret_cast<const V*>(a.out_u);
                const V* oY = reinterpret_cast<const V*>(a.out_u + g.N);
                for (int o = max(y0, g.probe_lo[1]); o < min(min(y0 + R, ny), g.probe_hi[1]); ++o) {
                    if (wall_side(o, ny, g.periodic[1]) >= 0) continue;
                    const int go = o * half + (xe >> 1);
                    const V ux = oX[go], uy = oY[go];
                    if (pxe && wxe < 0) {
                        const T nu = a.dir[0] * ux.x + a.dir[1] * uy.x;
                        jacc += nu;
                        qacc += nu * nu;
                    }
                    if (pxo && wxo < 0) {
                        const T nu = a.dir[0] * ux.y + a.dir[1] * uy.y;
                        jacc += nu;
                        qacc += nu * nu;
                    }
                }
            }
            store_probe_partials<32 * WY, T>(jacc, qacc, a.jslot, a.jsq, bx + a.jb_n[0] * by, red);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1}, recording lam_u and u_n on the footprint box.
// Each lane fetches its own data (its column pair of the source row's lambda, the source row's 1/(1 + kappa) on
// footprint rows, u_{n-1} and on footprint rows u_n of the output row) by asynchronous copies into a per-warp ring of
// Adj2vRing::DEPTH rows in shared memory, DEPTH - 1 rows ahead of use, so that many rows are in flight without holding
// them in registers; a lane reads back only what it copied, so the ring needs no barrier.  The row's
// uniform work (wrap, wall test, footprint row) is done once per row.  Indices are 32-bit (offered when 3 N and
// 4 F_b fit).
// ------------------------------------------------------------------------------------------------
template <typename T>
struct Adj2vRing {
    static constexpr int WY = 4;                               // warps per block
    static constexpr int DEPTH = sizeof(T) == 4 ? 6 : 3;       // rows per warp ring
    using V = typename Vec2<T>::type;
    // per row and lane: lambda p, x, y and u_{n-1} x, y, u_n x, y (V each), then the factor pair (T each)
    static constexpr size_t ROW_V = 7 * 32, ROW_T = 2 * 32;
    static constexpr size_t bytes() { return (size_t)WY * DEPTH * (ROW_V * sizeof(V) + ROW_T * sizeof(T)); }
};

template <typename T, int HW, int R>
__global__ void __launch_bounds__(128, 4) adj2v_kernel(Geom g, AdjArgs<T> a) {
    using V = typename Vec2<T>::type;
    using RG = Adj2vRing<T>;
    constexpr int WY = RG::WY, DEPTH = RG::DEPTH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V* rv = reinterpret_cast<V*>(smem_raw) + (size_t)warp * DEPTH * RG::ROW_V;                  // [DEPTH][7][32]
    T* rt = reinterpret_cast<T*>(reinterpret_cast<V*>(smem_raw) + (size_t)WY * DEPTH * RG::ROW_V) +
            (size_t)warp * DEPTH * RG::ROW_T;                                                      // [DEPTH][2][32]
    const int nx = g.n[0], ny = g.n[1];
    const int N = (int)g.N, Fbn = (int)g.Fbn, Fb0 = g.Fb[0];
    const int x0 = blockIdx.x * kVecCols;
    const int y0 = (blockIdx.y * WY + warp) * R;
    const int xe = x0 - 2 + 2 * lane;
    const int xl = wrap(xe, nx);
    const bool lane_out = lane >= 1 && lane <= 30 && xe < nx;
    const T A = (T)g.A;
    const V* __restrict__ lP = reinterpret_cast<const V*>(a.lam_in);
    const V* __restrict__ lX = reinterpret_cast<const V*>(a.lam_in + N);
    const V* __restrict__ lY = reinterpret_cast<const V*>(a.lam_in + 2 * N);
    const V* __restrict__ upX = reinterpret_cast<const V*>(a.u_prev);
    const V* __restrict__ upY = reinterpret_cast<const V*>(a.u_prev + N);
    const V* __restrict__ ucX = reinterpret_cast<const V*>(a.u_cur);
    const V* __restrict__ ucY = reinterpret_cast<const V*>(a.u_cur + N);
    const Pose& P = *a.pose;
    const int half = nx >> 1;
    // per-lane invariants: source columns (wrapped) and output columns
    const int sbxe = box_coord(xl, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int sbxo = box_coord(xl + 1, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const bool swxe = wall_side(xl, nx, g.periodic[0]) >= 0, swxo = wall_side(xl + 1, nx, g.periodic[0]) >= 0;
    const int bxe = box_coord(xe, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const int bxo = box_coord(xe + 1, P.xs[0], g.Fb[0], nx, g.periodic[0]);
    const bool wxe = wall_side(xe, nx, g.periodic[0]) >= 0, wxo = wall_side(xe + 1, nx, g.periodic[0]) >= 0;
    const bool pxe = xe >= g.probe_lo[0] && xe < g.probe_hi[0];
    const bool pxo = xe + 1 >= g.probe_lo[0] && xe + 1 < g.probe_hi[0];
    const T one = (T)1, zr = (T)0;
    constexpr int NRW = R + 4;  // source rows y0 - 2 .. y0 + R + 1; row t is source row y0 - 2 + t, output row y0 - 4 + t
    pdl_wait_then_release();

    // copy group t: source row r = y0 - 2 + t (lambda; factors on footprint rows) and output row z = r - 2 (u_{n-1};
    // u_n on footprint rows), into ring slot t mod DEPTH
    auto issue = [&](int t) {
        if (t < NRW) {
            V* sv = rv + (t % DEPTH) * RG::ROW_V;
            T* st = rt + (t % DEPTH) * RG::ROW_T;
            const int yw = wrap(y0 - 2 + t, ny);
            const int gi = yw * half + (xl >> 1);
            cp_async<sizeof(V)>(sv + lane, lP + gi);
            cp_async<sizeof(V)>(sv + 32 + lane, lX + gi);
            cp_async<sizeof(V)>(sv + 64 + lane, lY + gi);
            if (a.fac != nullptr && wall_side(yw, ny, g.periodic[1]) < 0) {
                const int by = box_coord(yw, P.xs[1], g.Fb[1], ny, g.periodic[1]);
                if (by >= 0) {
                    const T* fr = a.fac + by * Fb0;
                    if (sbxe >= 0) cp_async<sizeof(T)>(st + lane, fr + sbxe);
                    if (sbxo >= 0) cp_async<sizeof(T)>(st + 32 + lane, fr + sbxo);
                }
            }
            const int z = y0 - 4 + t;
            if (t >= 4 && lane_out && z < ny && z < y0 + R) {
                const int gz = z * half + (xe >> 1);
                cp_async<sizeof(V)>(sv + 96 + lane, upX + gz);
                cp_async<sizeof(V)>(sv + 128 + lane, upY + gz);
                if (box_coord(z, P.xs[1], g.Fb[1], ny, g.periodic[1]) >= 0 && (bxe >= 0 || bxo >= 0)) {
                    cp_async<sizeof(V)>(sv + 160 + lane, ucX + gz);
                    cp_async<sizeof(V)>(sv + 192 + lane, ucY + gz);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < DEPTH - 1; ++t) issue(t);

    // moment accumulators as (even, odd) pairs of four rows that take the roles r-2 (completed, output), r-1, r and
    // r+1 in turn: the loop body is unrolled four times with the roles renamed, instead of moving the sets between
    // registers every row; xyp, yyp keep M2_xy and M2_yy of row r-3
    struct Mom { V m0, mx, my, xx, xy, yy; };
    const V zero = vsplat<T>(0.0);
    Mom S0{zero, zero, zero, zero, zero, zero}, S1 = S0, S2 = S0, S3 = S0;
    V xyp = zero, yyp = zero;
    const V c3 = vsplat<T>(3.0), c9 = vsplat<T>(9.0), cm3 = vsplat<T>(-3.0), vA = vmk(A, A);
    // raw lam_u of the source rows r-1 and r-2 (the output row's footprint record); the ring slot of row r-2 is
    // being refilled by then
    V rx1 = zero, ry1 = zero, rx2 = zero, ry2 = zero;

    // row t: ac = row r-2, a0 = row r-1, a1 = row r, a2 = row r+1 (r = y0 - 2 + t)
    auto step = [&](int t, Mom& ac, Mom& a0, Mom& a1, Mom& a2) {
        issue(t + DEPTH - 1);  // into the slot of row t - 1, read in the previous iteration
        cp_async_wait<DEPTH - 1>();  // this lane's copies of row t have landed
        const int r = y0 - 2 + t;
        const V* sv = rv + (t % DEPTH) * RG::ROW_V;
        const T* st = rt + (t % DEPTH) * RG::ROW_T;
        const V lp = sv[lane], lxv = sv[32 + lane], lyv = sv[64 + lane];
        // source row r: p-bar*/3 = lam_p / 3, u-bar* = lam_u * factor (1/(1 + kappa) off the walls, 0 on them)
        V fac;
        {
            const int yw = wrap(r, ny);
            T fe = one, fo = one;
            if (wall_side(yw, ny, g.periodic[1]) >= 0) {
                fe = fo = zr;
            } else {
                const int by = box_coord(yw, P.xs[1], g.Fb[1], ny, g.periodic[1]);
                if (by >= 0) {
                    if (a.fac != nullptr) {
                        if (sbxe >= 0) fe = st[lane];
                        if (sbxo >= 0) fo = st[32 + lane];
                    } else {
                        if (sbxe >= 0) {
                            const int b[2] = {sbxe, by};
                            fe = adj_inv<T, 2, HW>(g, P, a.kref, nullptr, b);
                        }
                        if (sbxo >= 0) {
                            const int b[2] = {sbxo, by};
                            fo = adj_inv<T, 2, HW>(g, P, a.kref, nullptr, b);
                        }
                    }
                }
                if (swxe) fe = zr;
                if (swxo) fo = zr;
            }
            fac = vmk(fe, fo);
        }
        const V P3 = vmul(vsplat<T>(1.0 / 3.0), lp), U = vmul(lxv, fac), W = vmul(lyv, fac);
        // sources x-1 of the pair (previous lane's odd, even) and x+1 (odd, next lane's even)
        const V P3L = vmk(shfl_u(P3.y), P3.x), P3R = vmk(P3.y, shfl_d(P3.x));
        const V UL = vmk(shfl_u(U.y), U.x), UR = vmk(U.y, shfl_d(U.x));
        const V WL = vmk(shfl_u(W.y), W.x), WR = vmk(W.y, shfl_d(W.x));
        const V FL0 = vsub(P3L, UL), FR0 = vadd(P3R, UR);  // F-bar of the sources at x-1, x+1 with c_y = 0
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            // F-bar_i(y) = p-bar*(y + c_i)/3 + c_i . u-bar*(y + c_i) for c = (-1, cy), (0, cy), (1, cy)
            const V FL = cy == 0 ? FL0 : vfma(vsplat<T>(cy), WL, FL0);
            const V FC = cy == 0 ? P3 : vfma(vsplat<T>(cy), W, P3);
            const V FR = cy == 0 ? FR0 : vfma(vsplat<T>(cy), WR, FR0);
            const double Wy = cy == 0 ? 2.0 / 3.0 : 1.0 / 6.0;
            const V Sx = vmul(vsplat<T>(Wy / 6.0), vadd(FL, FR));
            const V S = vfma(vsplat<T>(Wy * 2.0 / 3.0), FC, Sx), D = vmul(vsplat<T>(Wy / 6.0), vsub(FR, FL));
            if (cy == 1) {  // moment row r-1
                a0.m0 = vadd(a0.m0, S); a0.mx = vadd(a0.mx, D); a0.my = vadd(a0.my, S);
                a0.xx = vadd(a0.xx, Sx); a0.xy = vadd(a0.xy, D); a0.yy = vadd(a0.yy, S);
            } else if (cy == 0) {  // row r
                a1.m0 = vadd(a1.m0, S); a1.mx = vadd(a1.mx, D); a1.xx = vadd(a1.xx, Sx);
            } else {  // row r+1
                a2.m0 = vadd(a2.m0, S); a2.mx = vadd(a2.mx, D); a2.my = vsub(a2.my, S);
                a2.xx = vadd(a2.xx, Sx); a2.xy = vsub(a2.xy, D); a2.yy = vadd(a2.yy, S);
            }
        }
        // lambda_{n-1} of row z = r - 2 from moment rows z-1 (p), z (ac), z+1 (a0)
        const int z = r - 2;
        if (z >= y0) {
            const V xxL = vmk(shfl_u(ac.xx.y), ac.xx.x), xxR = vmk(ac.xx.y, shfl_d(ac.xx.x));
            const V xyL = vmk(shfl_u(ac.xy.y), ac.xy.x), xyR = vmk(ac.xy.y, shfl_d(ac.xy.x));
            if (lane_out && z < ny) {
                const V u0 = sv[96 + lane], u1 = sv[128 + lane];
                const int go = z * half + (xe >> 1);
                // lam_u' = 3 M1 - 3 u M0 + 9 M2 u + A sum_a [M2_a.(z - e_a) - M2_a.(z + e_a)]
                V vx = vmul(c9, vfma(ac.xy, u1, vmul(ac.xx, u0)));
                V vy = vmul(c9, vfma(ac.yy, u1, vmul(ac.xy, u0)));
                vx = vfma(c3, ac.mx, vfma(vmul(cm3, u0), ac.m0, vx));
                vy = vfma(c3, ac.my, vfma(vmul(cm3, u1), ac.m0, vy));
                vx = vfma(vA, vadd(vsub(xxL, xxR), vsub(xyp, a0.xy)), vx);
                vy = vfma(vA, vadd(vsub(xyL, xyR), vsub(yyp, a0.yy)), vy);
                const bool wy = wall_side(z, ny, g.periodic[1]) >= 0;
                const bool we = wy || wxe, wo = wy || wxo;
                if (a.src && z >= g.probe_lo[1] && z < g.probe_hi[1]) {
                    if (pxe && !we) {
                        const T f = src_factor(a, a.dir[0] * u0.x + a.dir[1] * u1.x);
                        vx.x += a.phi_dir[0] * f;
                        vy.x += a.phi_dir[1] * f;
                    }
                    if (pxo && !wo) {
                        const T f = src_factor(a, a.dir[0] * u0.y + a.dir[1] * u1.y);
                        vx.y += a.phi_dir[0] * f;
                        vy.y += a.phi_dir[1] * f;
                    }
                }
                V* oP = reinterpret_cast<V*>(a.lam_out);
                V* oX = reinterpret_cast<V*>(a.lam_out + N);
                V* oY = reinterpret_cast<V*>(a.lam_out + 2 * N);
                oP[go] = vmul(c3, ac.m0);
                oX[go] = vx;
                oY[go] = vy;
                const int by = box_coord(z, P.xs[1], g.Fb[1], ny, g.periodic[1]);
                if (by >= 0 && (bxe >= 0 || bxo >= 0)) {
                    // records: raw lam_u of row z (0 on walls) and u_n
                    const V c0 = sv[160 + lane], c1 = sv[192 + lane];
                    const int bl = by * Fb0;
                    if (bxe >= 0) {
                        a.boxbuf[bl + bxe] = we ? zr : rx2.x;
                        a.boxbuf[Fbn + bl + bxe] = we ? zr : ry2.x;
                        a.boxbuf[2 * Fbn + bl + bxe] = c0.x;
                        a.boxbuf[3 * Fbn + bl + bxe] = c1.x;
                    }
                    if (bxo >= 0) {
                        a.boxbuf[bl + bxo] = wo ? zr : rx2.y;
                        a.boxbuf[Fbn + bl + bxo] = wo ? zr : ry2.y;
                        a.boxbuf[2 * Fbn + bl + bxo] = c0.y;
                        a.boxbuf[3 * Fbn + bl + bxo] = c1.y;
                    }
                }
            }
        }
        // the completed row's M2_xy, M2_yy become row r-3's for the next row; its set starts row r+2 from zero
        xyp = ac.xy;
        yyp = ac.yy;
        ac = Mom{zero, zero, zero, zero, zero, zero};
        rx2 = rx1; ry2 = ry1; rx1 = lxv; ry1 = lyv;
    };
    static_assert(NRW % 4 == 0, "rows come in fours");
#pragma unroll 1
    for (int t = 0; t < NRW; t += 4) {
        step(t, S0, S1, S2, S3);
        step(t + 1, S1, S2, S3, S0);
        step(t + 2, S2, S3, S0, S1);
        step(t + 3, S3, S0, S1, S2);
    }
    cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------------------
// The footprint-box side of the reverse sweep for the FP32 state and the hat kernel (D2Q9).
// ------------------------------------------------------------------------------------------------
// 1 / (1 + kappa) over the footprint box for steps n_first .. n_first + nsteps - 1 (box_fac_kernel) with map_hat2,
// the arithmetic of the forward step, which writes the same factors for the steps it recomputes.
static __global__ void __launch_bounds__(256) box_fac_hat2_kernel(Geom g, const Pose* __restrict__ poses,
                                                                  const float* __restrict__ kref, int n_first,
                                                                  float* __restrict__ fac) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    const int j = blockIdx.y;
    int b[3];
    box_unflatten<2>(g, bl, b);
    float kap, C;
    map_hat2(g, poses[n_first + j], kref, b[0], b[1], kap, C);
    fac[j * g.Fbn + bl] = __fdiv_rn(1.f, __fadd_rn(1.f, kap));
}

// Local shape and motion sensitivities of a segment (adj_sens_kernel's quantities, Eqs. dJdgamma, dJdchi in discrete
// form): one thread per (footprint-box column bx, chunk of kSensHat2YC rows, step) marching up its chunk.  Per design
// row jy the two x taps give K(jy) = sum w_x kappa^ref and X(jy) = sum w'_x kappa^ref (w' = dw/d offset), and at box
// row by, whose y taps are jy = by - 1 and by,
//   kappa = sum w_y K,   dkappa/ds = (sum w_y X, sum w'_y K),   C = S_x S_y,   dC/ds = (S'_x S_y, S_x S'_y)
// with S, S' the sums of the valid weights and of their derivatives.  The loads of four rows are issued before they
// are used.  Motion partials: FP32 over the chunk and the block (fixed order), FP64 from the block sums on (blocks:
// the column blocks of the first chunk, then of the next...).  kappa-bar goes to kbar (0 outside the grid).
constexpr int kSensHat2NT = 128, kSensHat2YC = 16;

static __global__ void __launch_bounds__(kSensHat2NT)
    adj_sens_hat2_kernel(Geom g, const Pose* __restrict__ poses, const float* __restrict__ kref,
                         const float* __restrict__ boxbuf, long long bstride, int n_first, float* __restrict__ kbar,
                         double* __restrict__ mslot) {
    __shared__ double red[4 * (kSensHat2NT / 32)];
    const int s = blockIdx.y;
    const Pose& P = poses[n_first + s];
    const int fb0 = g.Fb[0];
    const long long Fbn = g.Fbn;
    const int ncb = (fb0 + kSensHat2NT - 1) / kSensHat2NT;  // column blocks per chunk
    const int bx = (blockIdx.x % ncb) * kSensHat2NT + threadIdx.x;
    const int by0 = (blockIdx.x / ncb) * kSensHat2YC, by1 = min(by0 + kSensHat2YC, g.Fb[1]);
    float mv[4] = {0.f, 0.f, 0.f, 0.f};
    const bool colin = bx < fb0;
    const bool ok = colin && (g.periodic[0] || (unsigned)(P.xs[0] + bx) < (unsigned)g.n[0]);
    float* kbo = colin && kbar != nullptr ? kbar + (long long)s * Fbn + bx : nullptr;
    if (!ok && kbo != nullptr) {
        for (int by = by0; by < by1; ++by) kbo[(long long)fb0 * by] = 0.f;
    }
    if (ok) {
        float wx[2], dwx[2], sx = 0.f, dsx = 0.f;
        int ix[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int jx = bx - 1 + k;
            const bool vx = jx >= 0 && jx < g.nde[0];
            wx[k] = vx ? P.wf[0][k] : 0.f;
            dwx[k] = vx ? P.dwf[0][k] : 0.f;
            ix[k] = vx ? jx : 0;
            sx += wx[k];
            dsx += dwx[k];
        }
        const float wy[2] = {P.wf[1][0], P.wf[1][1]}, dwy[2] = {P.dwf[1][0], P.dwf[1][1]};
        const float uG[2] = {P.uGf[0], P.uGf[1]};
        const int nde0 = g.nde[0], nde1 = g.nde[1], xs1 = P.xs[1], ny = g.n[1];
        const bool yper = g.periodic[1] != 0;
        const float* rec = boxbuf + (long long)s * bstride + bx;
        // the two x taps of design row jy (0 off the design grid)
        auto taps = [&](int jy, float (&kr)[2]) {
            const bool v = jy >= 0 && jy < nde1;
            const float* kp = kref + (long long)nde0 * (v ? jy : 0);
#pragma unroll
            for (int t = 0; t < 2; ++t) kr[t] = v ? kp[ix[t]] : 0.f;
        };
        float K0, X0;  // x sums of design row by - 1
        {
            float kr[2];
            taps(by0 - 1, kr);
            K0 = wx[0] * kr[0] + wx[1] * kr[1];
            X0 = dwx[0] * kr[0] + dwx[1] * kr[1];
        }
        constexpr int U = 4;
#pragma unroll 1
        for (int bq = by0; bq < by1; bq += U) {
            float kr[U][2], rl[U][4];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int by = bq + u;
                in[u] = by < by1 && (yper || (unsigned)(xs1 + by) < (unsigned)ny);
                taps(by < by1 ? by : -1, kr[u]);
                const long long o = (long long)fb0 * (in[u] ? by : 0);
#pragma unroll
                for (int c = 0; c < 4; ++c) rl[u][c] = in[u] ? rec[c * Fbn + o] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int by = bq + u;
                const float K1 = wx[0] * kr[u][0] + wx[1] * kr[u][1];  // design row by
                const float X1 = dwx[0] * kr[u][0] + dwx[1] * kr[u][1];
                if (in[u]) {
                    const bool v0 = by >= 1, v1 = by < nde1;  // y taps jy = by - 1, by on the design grid
                    const float wy0 = v0 ? wy[0] : 0.f, wy1 = v1 ? wy[1] : 0.f;
                    const float dy0 = v0 ? dwy[0] : 0.f, dy1 = v1 ? dwy[1] : 0.f;
                    const float kap = wy0 * K0 + wy1 * K1;
                    const float dk[2] = {wy0 * X0 + wy1 * X1, dy0 * K0 + dy1 * K1};
                    const float sy = wy0 + wy1, dsy = dy0 + dy1;
                    const float C = sx * sy;
                    const float dC[2] = {dsx * sy, sx * dsy};
                    const float inv = 1.f / (1.f + kap);
                    float kb = 0.f, cbar = 0.f, usb[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float lu = rl[u][c];
                        kb += lu * (uG[c] * C - rl[u][2 + c]);
                        usb[c] = lu * kap * inv;
                        cbar += usb[c] * uG[c];
                    }
                    kb *= inv;
                    if (kbo != nullptr) kbo[(long long)fb0 * by] = kb;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        mv[c] += kb * dk[c] + cbar * dC[c];
                        mv[2 + c] += usb[c] * C;
                    }
                } else if (by < by1 && kbo != nullptr) {
                    kbo[(long long)fb0 * by] = 0.f;
                }
                K0 = K1;
                X0 = X1;
            }
        }
    }
    if (mslot != nullptr) {
        double out[4];
        block_sum<kSensHat2NT, 4, float>(mv, out, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) mslot[((long long)s * gridDim.x + blockIdx.x) * 4 + c] = out[c];
        }
    }
}

// Transposed mapping onto the design grid (design_gather_kernel) for the FP32 state and the hat kernel: kappa-bar is
// 0 at footprint-box nodes outside the grid, so a tap needs no grid test, only to lie in the box (fixed per design
// node); the four tap-weight products of each step are staged once per block in shared memory, and each thread adds
// its steps' sums to its FP64 running sum in strict step order n = Nt..1 (across calls too).
constexpr int kGatherHat2NT = 128, kGatherHat2SC = 64;

static __global__ void __launch_bounds__(kGatherHat2NT)
    design_gather_hat2_kernel(Geom g, const Pose* __restrict__ poses, const float* __restrict__ kbar, int n_first,
                              int nsteps, long long kstride, double* __restrict__ dkref) {
    __shared__ float wp[kGatherHat2SC][4];
    const int nd = g.nde[0] * g.nde[1];
    const int jl = blockIdx.x * kGatherHat2NT + threadIdx.x;
    const bool act = jl < nd;
    const int jx = jl % g.nde[0], jy = jl / g.nde[0];
    // tap t = kx + 2 ky reads box node (j + 1 - k) per axis
    int off[4];
    bool val[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int bx = jx + 1 - (t & 1), by = jy + 1 - (t >> 1);
        val[t] = act && bx >= 0 && bx < g.Fb[0] && by >= 0 && by < g.Fb[1];
        off[t] = val[t] ? bx + g.Fb[0] * by : 0;
    }
    double acc = act ? dkref[jl] : 0.0;
    for (int c0 = nsteps - 1; c0 >= 0; c0 -= kGatherHat2SC) {
        const int cn = min(kGatherHat2SC, c0 + 1);  // steps c0, c0 - 1, .., c0 - cn + 1
        __syncthreads();
        for (int i = threadIdx.x; i < cn * 4; i += kGatherHat2NT) {
            const int u = i >> 2, t = i & 3;
            const Pose& P = poses[n_first + c0 - u];
            wp[u][t] = P.wf[0][t & 1] * P.wf[1][t >> 1];
        }
        __syncthreads();
        if (act) {
#pragma unroll 2
            for (int u = 0; u < cn; ++u) {
                const float* kb = kbar + (long long)(c0 - u) * kstride;
                float sum = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) sum = fmaf(wp[u][t], val[t] ? kb[off[t]] : 0.f, sum);
                acc += (double)sum;
            }
        }
    }
    if (act) dkref[jl] = acc;
}

}  // namespace lks
