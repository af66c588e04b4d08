// D2Q9 forward and adjoint step kernels on row tiles.
//
// A block of 32 x 8 threads owns an output tile 28 nodes wide and TY = 8 * RPT rows high.  Shared memory holds
// whole 32-lane rows (the tile plus a halo of 2 on each side), so every row is one coalesced warp load and a
// lane's x-neighbours are the adjacent words of the same row.  The forward stages the nine weighted equilibrium
// values w_i f_i of every node of the halo-1 region; the output node then reads the nine values that stream
// into it (one per direction).  The adjoint stages the nine values G_i = p-bar*/3 + c_i . u-bar* of every node of
// the halo-2 region, then the six local moments M0, M1, M2 of the halo-1 region.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"

namespace lks {

template <int RPT>
struct Row2 {
    static constexpr int W = 32, TXO = 28, TR = 8;      // row width, output columns, thread rows
    static constexpr int TY = TR * RPT;                  // output rows
    static constexpr int RR = TY + 4;                    // raw rows (halo 2)
    static constexpr int NT = W * TR;
};

template <typename T, int RPT>
__host__ __device__ constexpr size_t smem2r_fwd() {
    return sizeof(T) * (3 * Row2<RPT>::RR * 32 + 9 * Row2<RPT>::RR * 32);
}
template <typename T, int RPT>
__host__ __device__ constexpr size_t smem2r_adj() {
    return sizeof(T) * (9 * Row2<RPT>::RR * 32 + 6 * Row2<RPT>::RR * 32);
}

// Forward step n-1 -> n (Sec. 2.2 / 2.3), same arithmetic as fwd_step_kernel.
template <typename T, int HW, int RPT>
__global__ void __launch_bounds__(256) fwd2r_kernel(Geom g, FwdArgs<T> a) {
    using RW = Row2<RPT>;
    using L = Lattice<2>;
    constexpr int RR = RW::RR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[16];
    T* sp = reinterpret_cast<T*>(smem_raw);  // [RR][32] p'
    T* sx = sp + RR * 32;                    // u_x
    T* sy = sx + RR * 32;                    // u_y
    T* wf = sy + RR * 32;                    // [9][RR][32] weighted equilibrium values

    const int lane = threadIdx.x, t = threadIdx.y, tid = lane + 32 * t;
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * RW::TXO, y0 = blockIdx.y * RW::TY;
    const int xo = x0 + lane - 2;
    const int xl = wrap(xo, nx);
    const T A = (T)g.A;
    const Pose& P = *a.pose;
    // kappa and C of this thread's output nodes depend only on the pose and the design, not on the previous
    // step: evaluate them before waiting for it (programmatic dependent launch)
    const bool lane_out = lane >= 2 && lane <= 29 && xo < nx;
    const int bxc = box_coord(xo, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    T kapk[RPT], Ck[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int y = y0 + t + RW::TR * k;
        const int byc = box_coord(y, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        kapk[k] = 0;
        Ck[k] = 0;
        if (!g.rot && lane_out && y < ny && bxc >= 0 && byc >= 0) {
            const int b[2] = {bxc, byc};
            map_node<T, 2, HW, false>(g, P, a.kref, b, kapk[k], Ck[k], nullptr, nullptr);
        }
    }
    pdl_wait_then_release();
    // rotating body: kappa and u^S from the footprint map that the previous kernel wrote (so only after the wait)
    T uSk[RPT][2];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        uSk[k][0] = uSk[k][1] = 0;
        const int y = y0 + t + RW::TR * k;
        const int byc = box_coord(y, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        if (g.rot && lane_out && y < ny && bxc >= 0 && byc >= 0) {
            const T* map = (const T*)g.rotmap;
            const long long bl = bxc + (long long)g.Fb[0] * byc;
            kapk[k] = map[bl];
            uSk[k][0] = map[g.Fbn + bl];
            uSk[k][1] = map[2 * g.Fbn + bl];
        }
    }

    // phase 1: raw rows y0-2 .. y0+TY+1
#pragma unroll
    for (int r = t; r < RR; r += RW::TR) {
        const int gi = wrap(y0 - 2 + r, ny) * nx + xl;
        sp[r * 32 + lane] = a.in[gi];
        sx[r * 32 + lane] = a.in[g.N + gi];
        sy[r * 32 + lane] = a.in[2 * g.N + gi];
    }
    __syncthreads();
    // phase 2: w_i f_i on rows 1 .. RR-2, lanes 1 .. 30
    if (lane >= 1 && lane <= 30) {
        for (int m = 1 + t; m < RR - 1; m += RW::TR) {
            const int c = m * 32 + lane;
            const T p = sp[c], ux = sx[c], uy = sy[c];
            const T sig = (T)3 * p - (T)1.5 * (ux * ux + uy * uy);
            const T Txx = (T)4.5 * ux * ux + A * (sx[c + 1] - sx[c - 1]);
            const T Tyy = (T)4.5 * uy * uy + A * (sy[c + 32] - sy[c - 32]);
            const T Txy = (T)4.5 * ux * uy + (T)0.5 * A * ((sy[c + 1] - sy[c - 1]) + (sx[c + 32] - sx[c - 32]));
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int cx = L::c(q, 0), cy = L::c(q, 1);
                T f = sig;
                if (cx != 0) f += (T)(3 * cx) * ux + Txx;
                if (cy != 0) f += (T)(3 * cy) * uy + Tyy;
                if (cx * cy != 0) f += (T)(2 * cx * cy) * Txy;
                wf[q * RR * 32 + c] = (T)L::w(q) * f;
            }
        }
    }
    __syncthreads();
    // phase 3: outputs on rows 2 .. TY+1, lanes 2 .. 29
    T jacc = 0, qacc = 0;
    bool unstable = false;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int o = 2 + t + RW::TR * k;
        const int y = y0 - 2 + o;
        if (!lane_out || y >= ny) continue;
        const int c = o * 32 + lane;
        T fq[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) fq[q] = wf[q * RR * 32 + c - L::c(q, 0) - 32 * L::c(q, 1)];
        T accp = 0, ax = 0, ay = 0;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            accp += fq[q];
            if (L::c(q, 0) != 0) ax += (T)L::c(q, 0) * fq[q];
            if (L::c(q, 1) != 0) ay += (T)L::c(q, 1) * fq[q];
        }
        T un0 = ax, un1 = ay;
        const int byc = box_coord(y, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        if (bxc >= 0 && byc >= 0) {
            const T kap = kapk[k], C = Ck[k];
            const T inv = (T)1 / ((T)1 + kap);
            const T us0 = g.rot ? uSk[k][0] : pose_uG<T>(P, 0) * C, us1 = g.rot ? uSk[k][1] : pose_uG<T>(P, 1) * C;
            un0 = (ax + kap * us0) * inv;
            un1 = (ay + kap * us1) * inv;
        }
        int xg[2] = {xo, y};
        T uw[2];
        const bool wall = wall_node<T, 2>(g, xg, uw);
        if (wall) {
            un0 = uw[0];
            un1 = uw[1];
        }
        const long long go = (long long)y * nx + xo;
        a.out_p[go] = accp * (T)(1.0 / 3.0);
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
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int px = (int)blockIdx.x - a.jb_lo[0], py = (int)blockIdx.y - a.jb_lo[1];
        if (px >= 0 && px < a.jb_n[0] && py >= 0 && py < a.jb_n[1])
            store_probe_partials<256, T>(jacc, qacc, a.jslot, a.jsq, px + a.jb_n[0] * py, red);
    }
}

// Adjoint step lambda_n -> lambda_{n-1} (same algebra as adj_step_kernel), recording lam_u and u_n on the
// footprint box.
template <typename T, int HW, int RPT>
__global__ void __launch_bounds__(256) adj2r_kernel(Geom g, AdjArgs<T> a) {
    using RW = Row2<RPT>;
    using L = Lattice<2>;
    constexpr int RR = RW::RR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* gq = reinterpret_cast<T*>(smem_raw);  // [9][RR][32] G_i = p-bar*/3 + c_i . u-bar*
    T* mo = gq + 9 * RR * 32;                // [6][RR][32] M0, M1x, M1y, M2xx, M2yy, M2xy

    const int lane = threadIdx.x, t = threadIdx.y;
    const int nx = g.n[0], ny = g.n[1];
    const long long N = g.N;
    const int x0 = blockIdx.x * RW::TXO, y0 = blockIdx.y * RW::TY;
    const int xo = x0 + lane - 2;
    const int xl = wrap(xo, nx);
    const T A = (T)g.A;
    const Pose& P = *a.pose;
    const int bxl = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    // u_{n-1} (and u_n on the footprint box) of this thread's output nodes come from the forward recomputation,
    // complete before the previous step started: load them before waiting for it (programmatic dependent launch)
    const bool lane_out = lane >= 2 && lane <= 29 && xo < nx;
    const int bxc = box_coord(xo, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    T up0[RPT], up1[RPT], uc0[RPT], uc1[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int y = y0 + t + RW::TR * k;
        up0[k] = up1[k] = uc0[k] = uc1[k] = 0;
        if (lane_out && y < ny) {
            const long long go = (long long)y * nx + xo;
            up0[k] = a.u_prev[go];
            up1[k] = a.u_prev[N + go];
            if (bxc >= 0 && box_coord(y, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]) >= 0) {
                uc0[k] = a.u_cur[go];
                uc1[k] = a.u_cur[N + go];
            }
        }
    }
    pdl_wait_then_release();

    // phase 1: G_i of the source nodes of rows y0-2 .. y0+TY+1 (Brinkman and wall adjoint folded in)
#pragma unroll
    for (int r = t; r < RR; r += RW::TR) {
        const int yw = wrap(y0 - 2 + r, ny);
        const int gi = yw * nx + xl;
        const T lp = a.lam_in[gi];
        T ux = a.lam_in[N + gi], uy = a.lam_in[2 * N + gi];
        int xs[2] = {xl, yw};
        T uw[2];
        if (wall_node<T, 2>(g, xs, uw)) {
            ux = 0;
            uy = 0;
        } else {
            const int byl = box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
            if (bxl >= 0 && byl >= 0) {
                const int b[2] = {bxl, byl};
                const T inv = adj_inv<T, 2, HW>(g, P, a.kref, a.fac, b);
                ux *= inv;
                uy *= inv;
            }
        }
        const T p3 = lp * (T)(1.0 / 3.0);
        const int c = r * 32 + lane;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            T v = p3;
            if (L::c(q, 0) != 0) v += (T)L::c(q, 0) * ux;
            if (L::c(q, 1) != 0) v += (T)L::c(q, 1) * uy;
            gq[q * RR * 32 + c] = v;
        }
    }
    __syncthreads();
    // phase 2: moments of rows 1 .. RR-2, lanes 1 .. 30: M = sum_i w_i {1, c_i, c_i c_i} G_i(y + c_i)
    if (lane >= 1 && lane <= 30) {
        for (int m = 1 + t; m < RR - 1; m += RW::TR) {
            const int c = m * 32 + lane;
            T M0 = 0, M1x = 0, M1y = 0, Mxx = 0, Myy = 0, Mxy = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int cx = L::c(q, 0), cy = L::c(q, 1);
                const T v = (T)L::w(q) * gq[q * RR * 32 + c + cx + 32 * cy];
                M0 += v;
                if (cx != 0) {
                    M1x += (T)cx * v;
                    Mxx += v;
                }
                if (cy != 0) {
                    M1y += (T)cy * v;
                    Myy += v;
                }
                if (cx * cy != 0) Mxy += (T)(cx * cy) * v;
            }
            mo[c] = M0;
            mo[RR * 32 + c] = M1x;
            mo[2 * RR * 32 + c] = M1y;
            mo[3 * RR * 32 + c] = Mxx;
            mo[4 * RR * 32 + c] = Myy;
            mo[5 * RR * 32 + c] = Mxy;
        }
    }
    __syncthreads();
    // phase 3: lambda_{n-1} on rows 2 .. TY+1, lanes 2 .. 29
    const T* M0s = mo;
    const T* M1xs = mo + RR * 32;
    const T* M1ys = mo + 2 * RR * 32;
    const T* Mxxs = mo + 3 * RR * 32;
    const T* Myys = mo + 4 * RR * 32;
    const T* Mxys = mo + 5 * RR * 32;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int o = 2 + t + RW::TR * k;
        const int y = y0 - 2 + o;
        if (!lane_out || y >= ny) continue;
        const int c = o * 32 + lane;
        const long long go = (long long)y * nx + xo;
        const T u0 = up0[k], u1 = up1[k];
        const T M0 = M0s[c], Mxx = Mxxs[c], Myy = Myys[c], Mxy = Mxys[c];
        T vx = (T)3 * M1xs[c] - (T)3 * u0 * M0 + (T)9 * (Mxx * u0 + Mxy * u1) +
               A * ((Mxxs[c - 1] - Mxxs[c + 1]) + (Mxys[c - 32] - Mxys[c + 32]));
        T vy = (T)3 * M1ys[c] - (T)3 * u1 * M0 + (T)9 * (Mxy * u0 + Myy * u1) +
               A * ((Mxys[c - 1] - Mxys[c + 1]) + (Myys[c - 32] - Myys[c + 32]));
        int xg[2] = {xo, y};
        T uw[2];
        const bool wall = wall_node<T, 2>(g, xg, uw);
        if (a.src && !wall && in_probe<2>(g, xg)) {
            const T f = src_factor(a, a.dir[0] * u0 + a.dir[1] * u1);
            vx += a.phi_dir[0] * f;
            vy += a.phi_dir[1] * f;
        }
        a.lam_out[go] = (T)3 * M0;
        a.lam_out[N + go] = vx;
        a.lam_out[2 * N + go] = vy;
        const int byc = box_coord(y, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        if (bxc >= 0 && byc >= 0) {
            const long long bl = bxc + (long long)g.Fb[0] * byc;
            a.boxbuf[bl] = wall ? (T)0 : a.lam_in[N + go];
            a.boxbuf[g.Fbn + bl] = wall ? (T)0 : a.lam_in[2 * N + go];
            a.boxbuf[2 * g.Fbn + bl] = uc0[k];
            a.boxbuf[3 * g.Fbn + bl] = uc1[k];
        }
    }
}

}  // namespace lks

namespace lks {

struct Fused2 {
    static constexpr int TY = 8, RR = TY + 8, TXO = 24;
};
template <typename T>
__host__ __device__ constexpr size_t smem2r2_fwd() {
    return sizeof(T) * 12 * Fused2::RR * 32;
}

// Two forward steps n-1 -> n -> n+1 in one launch (D2Q9).  The tile is 24 columns wide (32-lane rows with a halo
// of 4) and 8 rows high; step n is computed on the tile plus a halo of 2, kept in shared memory as the input of
// step n+1, and written out for the tile itself.  The arithmetic per step is that of fwd2r_kernel.
// With two = 0 only step n is taken (the last step of an odd run), on the same tile geometry.
template <typename T, int HW, bool SQ>
__global__ void __launch_bounds__(256) fwd2r2_kernel(Geom g, FwdArgs<T> a1, FwdArgs<T> a2, int two) {
    using L = Lattice<2>;
    constexpr int TY = Fused2::TY, RR = Fused2::RR, TXO = Fused2::TXO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[SQ ? 16 : 8];
    T* sp = reinterpret_cast<T*>(smem_raw);  // [RR][32] p', then step-n state in place
    T* sx = sp + RR * 32;
    T* sy = sx + RR * 32;
    T* wf = sy + RR * 32;                    // [9][RR][32]

    const int lane = threadIdx.x, t = threadIdx.y, tid = lane + 32 * t;
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * TXO, y0 = blockIdx.y * TY;
    const int xo = x0 + lane - 4;           // this lane's column (may lie outside [0, nx))
    const int xl = wrap(xo, nx);
    const T A = (T)g.A;
    // kappa and C of this thread's output nodes of both steps (rows h + t + 8 m, h = 2 for step n and 4 for step
    // n+1) depend only on the poses and the design: evaluate them before waiting for the previous step
    T kap1[2], C1[2], kap2[2], C2[2];
    auto premap = [&](int h, const FwdArgs<T>& a, T* kk, T* cc, int nrow) {
        const Pose& P = *a.pose;
        const int bxc = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        for (int m = 0; m < nrow; ++m) {
            const int o = h + t + 8 * m;
            kk[m] = 0;
            cc[m] = 0;
            const int byc = box_coord(wrap(y0 - 4 + o, ny), P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
            if (lane >= h && lane < 32 - h && o < RR - h && bxc >= 0 && byc >= 0) {
                const int b[2] = {bxc, byc};
                map_node<T, 2, HW, false>(g, P, a.kref, b, kk[m], cc[m], nullptr, nullptr);
            }
        }
    };
    premap(2, a1, kap1, C1, 2);
    if (two) premap(4, a2, kap2, C2, 2);
    pdl_wait_then_release();

#pragma unroll
    for (int r = t; r < RR; r += 8) {
        const int gi = wrap(y0 - 4 + r, ny) * nx + xl;
        sp[r * 32 + lane] = a1.in[gi];
        sx[r * 32 + lane] = a1.in[g.N + gi];
        sy[r * 32 + lane] = a1.in[2 * g.N + gi];
    }
    __syncthreads();

    auto equilibria = [&](int h) {  // w_i f_i on rows [h, RR-h), lanes [h, 32-h)
        if (lane >= h && lane < 32 - h) {
            for (int m = h + t; m < RR - h; m += 8) {
                const int c = m * 32 + lane;
                const T p = sp[c], ux = sx[c], uy = sy[c];
                const T sig = (T)3 * p - (T)1.5 * (ux * ux + uy * uy);
                const T Txx = (T)4.5 * ux * ux + A * (sx[c + 1] - sx[c - 1]);
                const T Tyy = (T)4.5 * uy * uy + A * (sy[c + 32] - sy[c - 32]);
                const T Txy = (T)4.5 * ux * uy + (T)0.5 * A * ((sy[c + 1] - sy[c - 1]) + (sx[c + 32] - sx[c - 32]));
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int cx = L::c(q, 0), cy = L::c(q, 1);
                    T f = sig;
                    if (cx != 0) f += (T)(3 * cx) * ux + Txx;
                    if (cy != 0) f += (T)(3 * cy) * uy + Tyy;
                    if (cx * cy != 0) f += (T)(2 * cx * cy) * Txy;
                    wf[q * RR * 32 + c] = (T)L::w(q) * f;
                }
            }
        }
    };
    // stream + Brinkman + walls of the nodes on rows [h, RR-h), lanes [h, 32-h); results to shared memory and,
    // for the tile itself, to global memory (with the objective partial and the stability check)
    T jacc1 = 0, jacc2 = 0, qacc1 = 0, qacc2 = 0;
    bool unstable = false;
    auto outputs = [&](int h, const FwdArgs<T>& a, T& jacc, T& qacc, const T* kk, const T* cc) {
        const Pose& P = *a.pose;
        const int bxc = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        const bool lane_in = lane >= h && lane < 32 - h;
        const bool lane_tile = lane >= 4 && lane < 28 && xo < nx;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int o = h + t + 8 * m;
            if (o >= RR - h || !lane_in) continue;
            const int c = o * 32 + lane;
            const int yw = wrap(y0 - 4 + o, ny);
            T fq[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) fq[q] = wf[q * RR * 32 + c - L::c(q, 0) - 32 * L::c(q, 1)];
            T accp = 0, ax = 0, ay = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                accp += fq[q];
                if (L::c(q, 0) != 0) ax += (T)L::c(q, 0) * fq[q];
                if (L::c(q, 1) != 0) ay += (T)L::c(q, 1) * fq[q];
            }
            T un0 = ax, un1 = ay;
            const int byc = box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
            if (bxc >= 0 && byc >= 0) {
                const T kap = kk[m], C = cc[m];
                const T inv = (T)1 / ((T)1 + kap);
                un0 = (ax + kap * (pose_uG<T>(P, 0) * C)) * inv;
                un1 = (ay + kap * (pose_uG<T>(P, 1) * C)) * inv;
            }
            int xg[2] = {xl, yw};
            T uw[2];
            const bool wall = wall_node<T, 2>(g, xg, uw);
            if (wall) {
                un0 = uw[0];
                un1 = uw[1];
            }
            const T pn = accp * (T)(1.0 / 3.0);
            // results of this step become the next step's input (this phase reads only wf)
            sp[c] = pn;
            sx[c] = un0;
            sy[c] = un1;
            const int y = y0 - 4 + o;
            if (lane_tile && o >= 4 && o < RR - 4 && y < ny) {
                const long long go = (long long)y * nx + xo;
                a.out_p[go] = pn;
                a.out_u[go] = un0;
                a.out_u[g.N + go] = un1;
                if (!wall) {
                    if (a.u_crit2 > (T)0 && !(un0 * un0 + un1 * un1 <= a.u_crit2)) unstable = true;
                    if (in_probe<2>(g, xg)) {
                        const T nu = a.dir[0] * un0 + a.dir[1] * un1;
                        jacc += nu;
                        if constexpr (SQ) qacc += nu * nu;
                    }
                }
            }
        }
    };
    equilibria(1);
    __syncthreads();
    outputs(2, a1, jacc1, qacc1, kap1, C1);
    if (two) {
        __syncthreads();
        equilibria(3);
        __syncthreads();
        outputs(4, a2, jacc2, qacc2, kap2, C2);
    }
    if (unstable) atomicOr(a1.flag, 1u);
    for (int s = 0; s < 1 + two; ++s) {
        const FwdArgs<T>& a = s == 0 ? a1 : a2;
        if (a.jslot == nullptr) continue;
        const int px = (int)blockIdx.x - a.jb_lo[0], py = (int)blockIdx.y - a.jb_lo[1];
        if (px >= 0 && px < a.jb_n[0] && py >= 0 && py < a.jb_n[1]) {
            __syncthreads();
            if constexpr (SQ) {
                store_probe_partials<256, T>(s == 0 ? jacc1 : jacc2, s == 0 ? qacc1 : qacc2, a.jslot, a.jsq,
                                             px + a.jb_n[0] * py, red);
            } else {
                T v[1] = {s == 0 ? jacc1 : jacc2};
                double sum[1];
                block_sum<256, 1, T>(v, sum, red);
                if (tid == 0) a.jslot[px + a.jb_n[0] * py] = sum[0];
            }
        }
    }
}

template <typename T>
__host__ __device__ constexpr size_t smem2r2_adj() {
    return sizeof(T) * 18 * Fused2::RR * 32;
}

// Two adjoint steps lambda_n -> lambda_{n-1} -> lambda_{n-2} in one launch (D2Q9), on the tile geometry of
// fwd2r2_kernel (24 x 8 outputs, 32-lane rows with a halo of 4).  Step n is computed on the tile plus a halo of
// 2 and kept in shared memory as the input of step n-1; lambda_{n-1} never goes to global memory.  Each step
// records lambda_u and u on the footprint box for the tile's own nodes.  The arithmetic per step is that of
// adj2r_kernel.  With two = 0 only step n is taken and its result written out (the last step of an odd run).
template <typename T, int HW>
__global__ void __launch_bounds__(256) adj2r2_kernel(Geom g, AdjArgs<T> a1, AdjArgs<T> a2, int two) {
    using L = Lattice<2>;
    constexpr int RR = Fused2::RR, TXO = Fused2::TXO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* gq = reinterpret_cast<T*>(smem_raw);  // [9][RR][32] G_i = p-bar*/3 + c_i . u-bar*
    T* mo = gq + 9 * RR * 32;                // [6][RR][32] M0, M1x, M1y, M2xx, M2yy, M2xy
    T* sl = mo + 6 * RR * 32;                // [3][RR][32] lambda_{n-1} (step n results)

    const int lane = threadIdx.x, t = threadIdx.y;
    const int nx = g.n[0], ny = g.n[1];
    const long long N = g.N;
    const int x0 = blockIdx.x * TXO, y0 = blockIdx.y * Fused2::TY;
    const int xo = x0 + lane - 4;
    const int xl = wrap(xo, nx);
    const T A = (T)g.A;
    const bool lane_tile = lane >= 4 && lane < 28 && xo < nx;
    // u_{n-1} and u_n of this thread's output nodes of both steps (rows h + t + 8 m, h = 2 for step n and 4 for
    // step n-1) come from the forward recomputation, complete before the previous launch started: load them
    // before waiting for it (u_n only where a footprint record is written)
    T up1[2][2], uc1[2][2], up2[2][2], uc2[2][2];
    auto preload = [&](int h, const AdjArgs<T>& a, T (*up)[2], T (*uc)[2]) {
        const Pose& P = *a.pose;
        const int bxc = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int o = h + t + 8 * m;
            up[m][0] = up[m][1] = uc[m][0] = uc[m][1] = 0;
            if (lane >= h && lane < 32 - h && o < RR - h) {
                const int yw = wrap(y0 - 4 + o, ny);
                const long long go = (long long)yw * nx + xl;
                up[m][0] = a.u_prev[go];
                up[m][1] = a.u_prev[N + go];
                const bool own = lane_tile && o >= 4 && o < RR - 4 && y0 - 4 + o < ny;
                if (own && bxc >= 0 && box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]) >= 0) {
                    uc[m][0] = a.u_cur[go];
                    uc[m][1] = a.u_cur[N + go];
                }
            }
        }
    };
    preload(2, a1, up1, uc1);
    if (two) preload(4, a2, up2, uc2);
    pdl_wait_then_release();

    // G_i of rows [h, RR-h), lanes [h, 32-h) from lambda (global for step n, shared memory for step n-1)
    auto stage = [&](int h, const AdjArgs<T>& a, bool from_smem) {
        const Pose& P = *a.pose;
        const int bxl = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        if (lane < h || lane >= 32 - h) return;
        for (int r = h + t; r < RR - h; r += 8) {
            const int yw = wrap(y0 - 4 + r, ny);
            const int c = r * 32 + lane;
            T lp, ux, uy;
            if (from_smem) {
                lp = sl[c];
                ux = sl[RR * 32 + c];
                uy = sl[2 * RR * 32 + c];
            } else {
                const long long gi = (long long)yw * nx + xl;
                lp = a.lam_in[gi];
                ux = a.lam_in[N + gi];
                uy = a.lam_in[2 * N + gi];
            }
            int xs[2] = {xl, yw};
            T uw[2];
            if (wall_node<T, 2>(g, xs, uw)) {
                ux = 0;
                uy = 0;
            } else {
                const int byl = box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
                if (bxl >= 0 && byl >= 0) {
                    const int b[2] = {bxl, byl};
                    const T inv = adj_inv<T, 2, HW>(g, P, a.kref, a.fac, b);
                    ux *= inv;
                    uy *= inv;
                }
            }
            const T p3 = lp * (T)(1.0 / 3.0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                T v = p3;
                if (L::c(q, 0) != 0) v += (T)L::c(q, 0) * ux;
                if (L::c(q, 1) != 0) v += (T)L::c(q, 1) * uy;
                gq[q * RR * 32 + c] = v;
            }
        }
    };
    // moments of rows [h, RR-h), lanes [h, 32-h)
    auto moments = [&](int h) {
        if (lane < h || lane >= 32 - h) return;
        for (int m = h + t; m < RR - h; m += 8) {
            const int c = m * 32 + lane;
            T M0 = 0, M1x = 0, M1y = 0, Mxx = 0, Myy = 0, Mxy = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int cx = L::c(q, 0), cy = L::c(q, 1);
                const T v = (T)L::w(q) * gq[q * RR * 32 + c + cx + 32 * cy];
                M0 += v;
                if (cx != 0) {
                    M1x += (T)cx * v;
                    Mxx += v;
                }
                if (cy != 0) {
                    M1y += (T)cy * v;
                    Myy += v;
                }
                if (cx * cy != 0) Mxy += (T)(cx * cy) * v;
            }
            mo[c] = M0;
            mo[RR * 32 + c] = M1x;
            mo[2 * RR * 32 + c] = M1y;
            mo[3 * RR * 32 + c] = Mxx;
            mo[4 * RR * 32 + c] = Myy;
            mo[5 * RR * 32 + c] = Mxy;
        }
    };
    // lambda_{n-1} of rows [h, RR-h), lanes [h, 32-h): to shared memory (to_smem) and, for the tile's own nodes,
    // to global memory (!to_smem); footprint-box records of the tile's own nodes
    auto outputs = [&](int h, const AdjArgs<T>& a, bool to_smem, bool lam_smem, const T (*up)[2], const T (*uc)[2]) {
        const Pose& P = *a.pose;
        const int bxc = box_coord(xl, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        const T* M0s = mo;
        const T* M1xs = mo + RR * 32;
        const T* M1ys = mo + 2 * RR * 32;
        const T* Mxxs = mo + 3 * RR * 32;
        const T* Myys = mo + 4 * RR * 32;
        const T* Mxys = mo + 5 * RR * 32;
        if (lane < h || lane >= 32 - h) return;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int o = h + t + 8 * m;
            if (o >= RR - h) continue;
            const int yw = wrap(y0 - 4 + o, ny);
            const int c = o * 32 + lane;
            const long long go = (long long)yw * nx + xl;
            const T u0 = up[m][0], u1 = up[m][1];
            const T M0 = M0s[c], Mxx = Mxxs[c], Myy = Myys[c], Mxy = Mxys[c];
            T vx = (T)3 * M1xs[c] - (T)3 * u0 * M0 + (T)9 * (Mxx * u0 + Mxy * u1) +
                   A * ((Mxxs[c - 1] - Mxxs[c + 1]) + (Mxys[c - 32] - Mxys[c + 32]));
            T vy = (T)3 * M1ys[c] - (T)3 * u1 * M0 + (T)9 * (Mxy * u0 + Myy * u1) +
                   A * ((Mxys[c - 1] - Mxys[c + 1]) + (Myys[c - 32] - Myys[c + 32]));
            int xg[2] = {xl, yw};
            T uw[2];
            const bool wall = wall_node<T, 2>(g, xg, uw);
            if (a.src && !wall && in_probe<2>(g, xg)) {
                const T f = src_factor(a, a.dir[0] * u0 + a.dir[1] * u1);
                vx += a.phi_dir[0] * f;
                vy += a.phi_dir[1] * f;
            }
            const bool own = lane_tile && o >= 4 && o < RR - 4 && y0 - 4 + o < ny;
            if (own) {
                // records of this step: lambda_n (the step's input) and u_n
                const int byc = box_coord(yw, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
                if (bxc >= 0 && byc >= 0) {
                    const long long bl = bxc + (long long)g.Fb[0] * byc;
                    const T lx = lam_smem ? sl[RR * 32 + c] : a.lam_in[N + go];
                    const T ly = lam_smem ? sl[2 * RR * 32 + c] : a.lam_in[2 * N + go];
                    a.boxbuf[bl] = wall ? (T)0 : lx;
                    a.boxbuf[g.Fbn + bl] = wall ? (T)0 : ly;
                    a.boxbuf[2 * g.Fbn + bl] = uc[m][0];
                    a.boxbuf[3 * g.Fbn + bl] = uc[m][1];
                }
            }
            if (to_smem) {
                // step n-1 reads sl only in its staging, which follows a barrier; the records above read the
                // step's own input, so sl is overwritten only in step n
                sl[c] = (T)3 * M0;
                sl[RR * 32 + c] = vx;
                sl[2 * RR * 32 + c] = vy;
            } else if (own) {
                a.lam_out[go] = (T)3 * M0;
                a.lam_out[N + go] = vx;
                a.lam_out[2 * N + go] = vy;
            }
        }
    };
    stage(0, a1, false);
    __syncthreads();
    moments(1);
    __syncthreads();
    outputs(2, a1, two != 0, false, up1, uc1);
    if (two) {
        __syncthreads();
        stage(2, a2, true);
        __syncthreads();
        moments(3);
        __syncthreads();
        outputs(4, a2, false, true, up2, uc2);
    }
}

}  // namespace lks
