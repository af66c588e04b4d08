// D3Q15 forward step in separable z-marching form.
//
// The streamed moments p* = (1/3) sum_i f_i(x - c_i) and u* = sum_i c_i f_i(x - c_i) of the LKS (Sec. 2.2) are
// linear in a handful of per-node fields once the equilibrium of Eq. feq is written as
//     f_i = w_i [ sigma + 3 c_i.u + c_i.T.c_i ],   sigma = 3p - 1.5|u|^2,   T = 4.5 u u + A (grad u + grad u^T)
// (central differences, A = 3/4 - 9 nu / 2).  For the 8 corner velocities c = (sx, sy, sz) the sum over the
// signs factors axis by axis into "sum" S g = g(-1) + g(+1) and "difference" D g = g(-1) - g(+1) operators on
// the fields Q = sigma + tr T, u and the off-diagonal T (a sign s_a of the velocity becomes a D along axis a).
// The x/y part of each product is formed from the four diagonal in-plane neighbours held in shared memory; the
// z part is a register recurrence along the column the thread marches: every plane emits its contribution to
// the planes below and above.  The 6 face velocities use the same S/D split with sigma + T_aa and u_a.  Per
// node this needs 6 stored fields and 36 shared-memory reads, against 15 stored weighted equilibria and 15
// reads in the direct form, and no equilibrium is evaluated on the halo more than once per plane.
//
// A block owns TX x TY columns and ZB planes; shared memory holds a ring of five raw planes (p', u on the
// halo-2 region, filled by asynchronous copies three planes ahead of use) and one plane of fields on the halo-1
// region.  Each thread evaluates the fields of its own
// column (kept in registers for the z recurrence) and at most one node of the halo-1 ring, carrying the
// velocity of the planes below and at its node in registers so that only in-plane neighbours come from
// shared memory.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"

namespace lks {

template <int TY_>
struct Sep3 {
    static constexpr int TX = 32, TY = TY_, NT = TX * TY;
    static constexpr int SX = TX + 4, SY = TY + 4, NS = SX * SY;  // halo-2 region (raw state)
    static constexpr int MX = TX + 2, MY = TY + 2, NM = MX * MY;  // halo-1 region (fields)
    static constexpr int NR = NM - NT;                            // halo-1 ring nodes
    static constexpr int PER = (NS + NT - 1) / NT;                // raw elements per thread and plane
    static_assert(NR <= NT, "one ring node per thread at most");
};

template <typename T, int TY>
__host__ __device__ constexpr size_t smem3s_fwd() {
    return sizeof(T) * (5 * 4 * Sep3<TY>::NS + 6 * Sep3<TY>::NM);
}

// Halo-1 coordinates (i, j) of ring node r: row j = 0, row j = MY - 1, column i = 0, column i = MX - 1.
template <int TY>
__device__ __forceinline__ void ring_node(int r, int& i, int& j) {
    using R = Sep3<TY>;
    if (r < R::MX) {
        i = r;
        j = 0;
    } else if (r < 2 * R::MX) {
        i = r - R::MX;
        j = R::MY - 1;
    } else if (r < 2 * R::MX + TY) {
        i = 0;
        j = r - 2 * R::MX + 1;
    } else {
        i = R::MX - 1;
        j = r - 2 * R::MX - TY + 1;
    }
}

// Forward step n-1 -> n (Sec. 2.2 / 2.3); same result as fwd_step_kernel up to the order of FP additions.
template <typename T, int HW, int ZB, int TY>
__global__ void __launch_bounds__(Sep3<TY>::NT, TY == 8 ? 3 : 1) fwd3s_kernel(Geom g, FwdArgs<T> a) {
    using R = Sep3<TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * (R::NT / 32)];
    T* raw = reinterpret_cast<T*>(smem_raw);  // [5 slots][p, ux, uy, uz][NS]
    T* fld = raw + 5 * 4 * R::NS;             // [Q, Txy, Txz, Tyz, phi_x, phi_y][NM]
    T* fQ = fld;
    T* fXY = fld + R::NM;
    T* fXZ = fld + 2 * R::NM;
    T* fYZ = fld + 3 * R::NM;
    T* fPX = fld + 4 * R::NM;
    T* fPY = fld + 5 * R::NM;

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const long long plane = (long long)nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const T A = (T)g.A, hA = (T)0.5 * (T)g.A;
    const T c45 = (T)4.5, c15 = (T)1.5;
    const Pose& P = *a.pose;

    long long off[R::PER];
#pragma unroll
    for (int e = 0; e < R::PER; ++e) {
        const int l = tid + e * R::NT;
        const int i = l % R::SX, j = l / R::SX;
        off[e] = (l < R::NS) ? (long long)wrap(x0 - 2 + i, nx) + (long long)nx * wrap(y0 - 2 + j, ny) : 0;
    }
    // field nodes of this thread: 0 = own column, 1 = a node of the halo-1 ring (tid < NR)
    const bool has1 = tid < R::NR;
    int fi[2], fj[2];
    fi[0] = tx + 1;
    fj[0] = ty + 1;
    ring_node<TY>(has1 ? tid : 0, fi[1], fj[1]);
    int mrow[2], rrow[2];  // index in the halo-1 and halo-2 regions
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        mrow[s] = fi[s] + R::MX * fj[s];
        rrow[s] = (fi[s] + 1) + R::SX * (fj[s] + 1);
    }
    pdl_wait_then_release();

    // raw planes arrive by asynchronous copies into a ring of five slots, three planes ahead of use (plane k in
    // slot (k - z0 + 2) mod 5): no registers hold them in flight and no shared-memory stores are issued for them
    auto slot_of = [&](int k) { return raw + ((k - z0 + 2) % 5) * 4 * R::NS; };
    auto issue = [&](int k) {
        T* dst = slot_of(k);
        const long long base = plane * wrap(k, nz);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            const int l = tid + e * R::NT;
            if (l < R::NS) {
#pragma unroll
                for (int f = 0; f < 4; ++f) cp_async<sizeof(T)>(dst + f * R::NS + l, a.in + f * N + base + off[e]);
            }
        }
        cp_async_commit();
    };
    issue(z0 - 2);
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    cp_async_wait<0>();
    __syncthreads();

    // velocity of the field nodes at the plane below (um) and at the plane (uc), and p' at the plane
    T um[2][3], uc[2][3], pc[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T* rb = slot_of(z0 - 2) + rrow[s];
        const T* rc = slot_of(z0 - 1) + rrow[s];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            um[s][c] = rb[(1 + c) * R::NS];
            uc[s][c] = rc[(1 + c) * R::NS];
        }
        pc[s] = rc[0];
    }

    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    // per-step pose values used on every plane, read once
    const int xs2 = P.xs[2];
    const T uG0 = pose_uG<T>(P, 0), uG1 = pose_uG<T>(P, 1), uG2 = pose_uG<T>(P, 2);
    const bool colbox = col && bx >= 0 && by >= 0;
    const T w0 = (T)(2.0 / 9.0), wf = (T)(1.0 / 9.0), wc = (T)(1.0 / 72.0), third = (T)(1.0 / 3.0);
    // partial streamed moments (p*, u*) of the plane below the current one and of the current plane
    T accM[4] = {0, 0, 0, 0}, accC[4] = {0, 0, 0, 0};
    bool unstable = false;

#pragma unroll 1
    for (int k = z0 - 1; k <= z0 + ZB; ++k) {
        // plane k + 3 into the slot of plane k - 2 (read last two iterations ago); plane k + 1 has arrived once
        // at most the two newest copy groups are pending (empty groups keep the count at the end of the run)
        if (k + 3 <= z0 + ZB + 1)
            issue(k + 3);
        else
            cp_async_commit();
        cp_async_wait<2>();
        __syncthreads();
        // (A) fields of plane k at the field nodes
        const T* rk = slot_of(k);
        const T* rn = slot_of(k + 1);
        T sig0 = 0, phz0 = 0, uz0 = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && !has1) break;
            const int r = rrow[s];
            T up[3], G[3][3];  // G[d][c]: twice the central difference of u_c along axis d
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T* f = rk + (1 + c) * R::NS;
                up[c] = rn[(1 + c) * R::NS + r];
                G[0][c] = f[r + 1] - f[r - 1];
                G[1][c] = f[r + R::SX] - f[r - R::SX];
                G[2][c] = up[c] - um[s][c];
            }
            const T ux = uc[s][0], uy = uc[s][1], uz = uc[s][2];
            const T sig = (T)3 * pc[s] - c15 * (ux * ux + uy * uy + uz * uz);
            const T Txx = c45 * ux * ux + A * G[0][0];
            const T Tyy = c45 * uy * uy + A * G[1][1];
            const T Tzz = c45 * uz * uz + A * G[2][2];
            const T Txy = c45 * ux * uy + hA * (G[0][1] + G[1][0]);
            const T Txz = c45 * ux * uz + hA * (G[0][2] + G[2][0]);
            const T Tyz = c45 * uy * uz + hA * (G[1][2] + G[2][1]);
            const int m = mrow[s];
            fQ[m] = sig + Txx + Tyy + Tzz;
            fXY[m] = Txy;
            fXZ[m] = Txz;
            fYZ[m] = Tyz;
            fPX[m] = sig + Txx;
            fPY[m] = sig + Tyy;
            if (s == 0) {
                sig0 = sig;
                phz0 = sig + Tzz;
                uz0 = uz;
            }
            // shift the z window: (k-1, k) <- (k, k+1)
            pc[s] = rn[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                um[s][c] = uc[s][c];
                uc[s][c] = up[c];
            }
        }
        __syncthreads();
        // (B) contributions of plane k to the moments of planes k-1, k, k+1 along this column
        {
            const int m = mrow[0];
            const int r = rrow[0];
            // corner terms: S/D products over the four diagonal in-plane neighbours
            // (a, b, c, d) = g at (x-1, y-1), (x+1, y-1), (x-1, y+1), (x+1, y+1)
            auto sd4 = [](const T* f, int i0, int sx, int sy, T& SS, T& DS, T& SD, T& DD) {
                const T va = f[i0 - 1 - sy], vb = f[i0 + 1 - sy], vc = f[i0 - 1 + sy], vd = f[i0 + 1 + sy];
                const T s1 = va + vb, s2 = vc + vd, d1 = va - vb, d2 = vc - vd;
                SS = s1 + s2;
                SD = s1 - s2;
                DS = d1 + d2;
                DD = d1 - d2;
                (void)sx;
            };
            T qSS, qDS, qSD, qDD, xSS, xDS, xSD, xDD, ySS, yDS, ySD, yDD, zSS, zDS, zSD, zDD;
            T aSS, aDS, aSD, aDD, bSS, bDS, bSD, bDD, cSS, cDS, cSD, cDD;
            sd4(fQ, m, 1, R::MX, qSS, qDS, qSD, qDD);
            sd4(rk + R::NS, r, 1, R::SX, xSS, xDS, xSD, xDD);
            sd4(rk + 2 * R::NS, r, 1, R::SX, ySS, yDS, ySD, yDD);
            sd4(rk + 3 * R::NS, r, 1, R::SX, zSS, zDS, zSD, zDD);
            sd4(fXY, m, 1, R::MX, aSS, aDS, aSD, aDD);
            sd4(fXZ, m, 1, R::MX, bSS, bDS, bSD, bDD);
            sd4(fYZ, m, 1, R::MX, cSS, cDS, cSD, cDD);
            const T A1 = qSS + (T)3 * (xDS + ySD) + (T)2 * aDD;
            const T A2 = (T)3 * zSS + (T)2 * (bDS + cSD);
            const T B1 = qDS + (T)3 * (xSS + yDD) + (T)2 * aSD;
            const T B2 = (T)3 * zDS + (T)2 * (bSS + cDD);
            const T C1 = qSD + (T)3 * (xDD + ySS) + (T)2 * aDS;
            const T C2 = (T)3 * zSD + (T)2 * (bDD + cSS);
            // face terms along x and y (in-plane) and along z (the column's own fields)
            const T* ux = rk + R::NS;
            const T* uy = rk + 2 * R::NS;
            const T pxm = fPX[m - 1], pxp = fPX[m + 1], pym = fPY[m - R::MX], pyp = fPY[m + R::MX];
            const T uxm = ux[r - 1], uxp = ux[r + 1], uym = uy[r - R::SX], uyp = uy[r + R::SX];
            const T inP = w0 * sig0 + wf * ((pxm + pxp) + (T)3 * (uxm - uxp) + (pym + pyp) + (T)3 * (uym - uyp));
            const T inX = wf * ((pxm - pxp) + (T)3 * (uxm + uxp));
            const T inY = wf * ((pym - pyp) + (T)3 * (uym + uyp));
            const T fzd = wf * (phz0 + (T)3 * uz0), fzu = wf * (phz0 - (T)3 * uz0);
            // emissions: to plane k+1 (this plane is its z-1 neighbour) and to plane k-1
            const T dnP = wc * (A1 + A2) + fzd, dnX = wc * (B1 + B2), dnY = wc * (C1 + C2), dnZ = wc * (A1 + A2) + fzd;
            const T upP = wc * (A1 - A2) + fzu, upX = wc * (B1 - B2), upY = wc * (C1 - C2), upZ = -(wc * (A1 - A2) + fzu);
            // plane k - 1 is complete
            accM[0] += upP;
            accM[1] += upX;
            accM[2] += upY;
            accM[3] += upZ;
            accC[0] += inP;
            accC[1] += inX;
            accC[2] += inY;
            const int zo = k - 1;
            if (zo >= z0 && zo < z0 + ZB && zo < nz && col) {
                const T pn = accM[0] * third;
                T un[3] = {accM[1], accM[2], accM[3]};
                int xyz[3] = {xg, yg, zo};
                const int bz = colbox ? box_coord(zo, xs2, g.Fb[2], g.n[2], g.periodic[2]) : -1;
                if (bz >= 0) {
                    const int b[3] = {bx, by, bz};
                    T kap, C;
                    map_node<T, 3, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
                    const T inv = (T)1 / ((T)1 + kap);
                    un[0] = (un[0] + kap * (uG0 * C)) * inv;
                    un[1] = (un[1] + kap * (uG1 * C)) * inv;
                    un[2] = (un[2] + kap * (uG2 * C)) * inv;
                }
                T uw[3];
                const bool wall = wall_node<T, 3>(g, xyz, uw);
                if (wall) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) un[c] = uw[c];
                }
                const long long gi = xg + (long long)nx * yg + plane * zo;
                a.out_p[gi] = pn;
#pragma unroll
                for (int c = 0; c < 3; ++c) a.out_u[c * N + gi] = un[c];
                if (!wall && a.u_crit2 > (T)0 && !(un[0] * un[0] + un[1] * un[1] + un[2] * un[2] <= a.u_crit2))
                    unstable = true;
            }
            // shift: plane k becomes the lower plane, plane k + 1 starts with this plane's emission
#pragma unroll
            for (int c = 0; c < 4; ++c) accM[c] = accC[c];
            accC[0] = dnP;
            accC[1] = dnX;
            accC[2] = dnY;
            accC[3] = dnZ;
        }
    }
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int px = (int)blockIdx.x - a.jb_lo[0], py = (int)blockIdx.y - a.jb_lo[1], pz = (int)blockIdx.z - a.jb_lo[2];
        if (px >= 0 && px < a.jb_n[0] && py >= 0 && py < a.jb_n[1] && pz >= 0 && pz < a.jb_n[2]) {
            // objective partials from this thread's own outputs, re-read after the march so that the march keeps
            // no accumulators (same nodes, planes upward)
            T jacc = 0, qacc = 0;
            if (col) {
                for (int zo = max(z0, g.probe_lo[2]); zo < min(min(z0 + ZB, nz), g.probe_hi[2]); ++zo) {
                    int xyz[3] = {xg, yg, zo};
                    T uw[3];
                    if (!in_probe<3>(g, xyz) || wall_node<T, 3>(g, xyz, uw)) continue;
                    const long long gi = xg + (long long)nx * yg + plane * zo;
                    const T nu = a.dir[0] * a.out_u[gi] + a.dir[1] * a.out_u[N + gi] + a.dir[2] * a.out_u[2 * N + gi];
                    jacc += nu;
                    qacc += nu * nu;
                }
            }
            store_probe_partials<R::NT, T>(jacc, qacc, a.jslot, a.jsq, px + a.jb_n[0] * (py + a.jb_n[1] * pz), red);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1} in separable z-marching form (same algebra as adj_step_kernel).
//
// The local moments M0 = sum_i w_i Fb_i, M1 = sum_i w_i c_i Fb_i, M2 = sum_i w_i c_i c_i Fb_i of
// Fb_i(y) = p-bar*(y + c_i) / 3 + c_i . u-bar*(y + c_i) are gathers from y + c_i, so for the corner velocities
// they factor into S g = g(+1) + g(-1) and D g = g(+1) - g(-1) products over the axes, exactly as in the
// forward step: with E0..E3 the xy products of (p-bar*/3, u-bar*_x, u-bar*_y) and Z0..Z3 those of u-bar*_z,
// a plane emits w (E + Z) to the plane below and w (E - Z) to the plane above.  Every halo-1 node of the block
// carries this z recurrence in registers; completed M2 planes go to a ring of three shared-memory planes, from
// which the A term (central differences of M2_ab along a) and the node's own M2 are read.  Output plane
// k - 2 is written while raw plane k is processed.
// ------------------------------------------------------------------------------------------------
template <typename T, int TY>
__host__ __device__ constexpr size_t smem3s_adj() {
    return sizeof(T) * (2 * 4 * Sep3<TY>::NS + 3 * 6 * Sep3<TY>::NM);
}

template <typename T, int HW, int ZB, int TY>
__global__ void __launch_bounds__(Sep3<TY>::NT, TY == 8 ? 3 : 1) adj3s_kernel(Geom g, AdjArgs<T> a) {
    using R = Sep3<TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* raw = reinterpret_cast<T*>(smem_raw);  // [2 slots][p-bar*/3, u-bar*_x, u-bar*_y, u-bar*_z][NS]
    T* mb = raw + 2 * 4 * R::NS;              // [3 planes][M2xx, M2yy, M2zz, M2xy, M2xz, M2yz][NM]

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const long long plane = (long long)nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const T A = (T)g.A;
    const Pose& P = *a.pose;
    const int xs2 = P.xs[2];

    // raw elements of this thread (halo-2 region): plane-invariant offsets, wall and footprint coordinates
    // (einner: the element is one of the block's own columns, whose footprint records it writes)
    long long off[R::PER];
    int ebx[R::PER], eby[R::PER];
    bool ewall[R::PER], einner[R::PER];
#pragma unroll
    for (int e = 0; e < R::PER; ++e) {
        const int l = tid + e * R::NT;
        const int i = l % R::SX, j = l / R::SX;
        const int ex = wrap(x0 - 2 + i, nx), ey = wrap(y0 - 2 + j, ny);
        off[e] = (l < R::NS) ? (long long)ex + (long long)nx * ey : 0;
        ebx[e] = box_coord(ex, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        eby[e] = box_coord(ey, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        ewall[e] = (!g.periodic[0] && (ex == 0 || ex == nx - 1)) || (!g.periodic[1] && (ey == 0 || ey == ny - 1));
        einner[e] = l < R::NS && i >= 2 && i < R::TX + 2 && j >= 2 && j < TY + 2 && x0 - 2 + i < nx && y0 - 2 + j < ny &&
                    ebx[e] >= 0 && eby[e] >= 0;
    }
    // field nodes: 0 = own column, 1 = a node of the halo-1 ring (tid < NR)
    const bool has1 = tid < R::NR;
    int fi[2], fj[2];
    fi[0] = tx + 1;
    fj[0] = ty + 1;
    ring_node<TY>(has1 ? tid : 0, fi[1], fj[1]);
    int mrow[2], rrow[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        mrow[s] = fi[s] + R::MX * fj[s];
        rrow[s] = (fi[s] + 1) + R::SX * (fj[s] + 1);
    }
    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const long long gcol = xg + (long long)nx * yg;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    const bool colbox = col && bx >= 0 && by >= 0;
    const bool wall_xy = (!g.periodic[0] && (xg == 0 || xg == nx - 1)) || (!g.periodic[1] && (yg == 0 || yg == ny - 1));
    const bool probe_xy = xg >= g.probe_lo[0] && xg < g.probe_hi[0] && yg >= g.probe_lo[1] && yg < g.probe_hi[1];
    pdl_wait_then_release();

    // lambda of a plane and, on the footprint box, its 1 / (1 + kappa), one plane ahead of use (this kernel
    // requires the box field a.fac)
    T pre[R::PER][4], pfac[R::PER];
    auto fetch = [&](int k) {
        const int kz = wrap(k, nz);
        const long long base = plane * kz;
        const int bz = box_coord(kz, xs2, g.Fb[2], g.n[2], g.periodic[2]);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            if (tid + e * R::NT < R::NS) {
#pragma unroll
                for (int f = 0; f < 4; ++f) pre[e][f] = a.lam_in[f * N + base + off[e]];
                pfac[e] = 1;
                if (ebx[e] >= 0 && eby[e] >= 0 && bz >= 0)
                    pfac[e] = a.fac[ebx[e] + (long long)g.Fb[0] * (eby[e] + (long long)g.Fb[1] * bz)];
            }
        }
    };
    // p-bar*/3 = lam_p / 3; u-bar* = lam_u / (1 + kappa), 0 on walls.  The lambda_u footprint records of the
    // block's own nodes are written here, from the raw lambda in registers.
    auto store = [&](int k, T* dst) {
        const int kz = wrap(k, nz);
        const bool wz = !g.periodic[2] && (kz == 0 || kz == nz - 1);
        const bool own_plane = k >= z0 && k < z0 + ZB && k < nz;
        const int bz = box_coord(kz, xs2, g.Fb[2], g.n[2], g.periodic[2]);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            const int l = tid + e * R::NT;
            if (l < R::NS) {
                const bool wall = ewall[e] || wz;
                const T fac = wall ? (T)0 : pfac[e];
                dst[l] = pre[e][0] * (T)(1.0 / 3.0);
#pragma unroll
                for (int f = 1; f < 4; ++f) dst[f * R::NS + l] = pre[e][f] * fac;
                if (einner[e] && own_plane && bz >= 0) {
                    const long long bl = ebx[e] + (long long)g.Fb[0] * (eby[e] + (long long)g.Fb[1] * bz);
#pragma unroll
                    for (int c = 0; c < 3; ++c) a.boxbuf[c * g.Fbn + bl] = wall ? (T)0 : pre[e][1 + c];
                }
            }
        }
    };
    T* sk = raw;               // slot of the plane being processed
    T* sn = raw + 4 * R::NS;   // slot of the next plane
    fetch(z0 - 2);
    store(z0 - 2, sk);
    fetch(z0 - 1);
    __syncthreads();

    const T w0 = (T)(2.0 / 9.0), wf = (T)(1.0 / 9.0), wc = (T)(1.0 / 72.0);
    // partial moments per field node, at the start of iteration k of planes k - 1 (C) and k (N):
    // M0, M1x, M1y, M1z, M2xx, M2yy, M2zz, M2xy, M2xz, M2yz
    T accC[2][10], accN[2][10];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int q = 0; q < 10; ++q) accC[s][q] = accN[s][q] = 0;
    T m0o = 0, m1o[3] = {0, 0, 0};  // own M0, M1 of the last completed plane
    T up0[3] = {0, 0, 0};           // u_{n-1} of the next output plane (prefetched)
    T uc0[3] = {0, 0, 0};           // u_n of the next output plane on the footprint box (prefetched)
    int mslot = 0;                  // M2 ring slot of plane k - 1

#pragma unroll 1
    for (int k = z0 - 2; k <= z0 + ZB + 1; ++k) {
        // own M0, M1 of plane k - 2 (completed in the previous iteration) for this iteration's output
        const T M0o = m0o, M1o0 = m1o[0], M1o1 = m1o[1], M1o2 = m1o[2];
        // (A) emissions of raw plane k; plane k - 1 completes
        T* mk1 = mb + mslot * 6 * R::NM;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && !has1) break;
            const int r = rrow[s];
            const T* fP = sk;
            const T* fX = sk + R::NS;
            const T* fY = sk + 2 * R::NS;
            const T* fZ = sk + 3 * R::NS;
            // S/D products over the diagonal neighbours; here D g = g(+1) - g(-1)
            T SS[4], DS[4], SD[4], DD[4];
            const T* fs[4] = {fP, fX, fY, fZ};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const T va = fs[f][r - 1 - R::SX], vb = fs[f][r + 1 - R::SX], vc = fs[f][r - 1 + R::SX],
                        vd = fs[f][r + 1 + R::SX];
                const T s1 = va + vb, s2 = vc + vd, d1 = vb - va, d2 = vd - vc;
                SS[f] = s1 + s2;
                SD[f] = s2 - s1;
                DS[f] = d1 + d2;
                DD[f] = d2 - d1;
            }
            const T E0 = SS[0] + DS[1] + SD[2], E1 = DS[0] + SS[1] + DD[2];
            const T E2 = SD[0] + DD[1] + SS[2], E3 = DD[0] + SD[1] + DS[2];
            const T U0 = wc * (E0 + SS[3]), U1 = wc * (E1 + DS[3]), U2 = wc * (E2 + SD[3]), U3 = wc * (E3 + DD[3]);
            const T L0 = wc * (E0 - SS[3]), L1 = wc * (E1 - DS[3]), L2 = wc * (E2 - SD[3]), L3 = wc * (E3 - DD[3]);
            // faces: in-plane x and y, and z from the node's own column
            const T pxm = fP[r - 1], pxp = fP[r + 1], vxm = fX[r - 1], vxp = fX[r + 1];
            const T pym = fP[r - R::SX], pyp = fP[r + R::SX], vym = fY[r - R::SX], vyp = fY[r + R::SX];
            const T pc = fP[r], vzc = fZ[r];
            const T fx = wf * ((pxp + pxm) + (vxp - vxm));   // M0 and M2xx part of the x faces
            const T fy = wf * ((pyp + pym) + (vyp - vym));
            const T zd = wf * (pc + vzc), zu = wf * (pc - vzc);  // to plane k - 1 and to plane k + 1
            T* cM = accC[s];
            T* nM = accN[s];
            // plane k - 1: complete it with the emission to the plane below
            const T c0 = cM[0] + U0 + zd, c1x = cM[1] + U1, c1y = cM[2] + U2, c1z = cM[3] + U0 + zd;
            const T c2xx = cM[4] + U0, c2yy = cM[5] + U0, c2zz = cM[6] + U0 + zd;
            const T c2xy = cM[7] + U3, c2xz = cM[8] + U1, c2yz = cM[9] + U2;
            const int m = mrow[s];
            mk1[m] = c2xx;
            mk1[R::NM + m] = c2yy;
            mk1[2 * R::NM + m] = c2zz;
            mk1[3 * R::NM + m] = c2xy;
            mk1[4 * R::NM + m] = c2xz;
            mk1[5 * R::NM + m] = c2yz;
            if (s == 0) {
                m0o = c0;
                m1o[0] = c1x;
                m1o[1] = c1y;
                m1o[2] = c1z;
            }
            // plane k: in-plane terms; plane k + 1: emission to the plane above
            cM[0] = nM[0] + w0 * pc + fx + fy;
            cM[1] = nM[1] + wf * ((pxp - pxm) + (vxp + vxm));
            cM[2] = nM[2] + wf * ((pyp - pym) + (vyp + vym));
            cM[3] = nM[3];
            cM[4] = nM[4] + fx;
            cM[5] = nM[5] + fy;
            cM[6] = nM[6];
            cM[7] = nM[7];
            cM[8] = nM[8];
            cM[9] = nM[9];
            nM[0] = L0 + zu;
            nM[1] = L1;
            nM[2] = L2;
            nM[3] = -(L0 + zu);
            nM[4] = L0;
            nM[5] = L0;
            nM[6] = L0 + zu;
            nM[7] = L3;
            nM[8] = -L1;
            nM[9] = -L2;
        }
        // raw plane k + 1 into the other slot, prefetch k + 2
        if (k + 1 <= z0 + ZB + 1) store(k + 1, sn);
        if (k + 2 <= z0 + ZB + 1) fetch(k + 2);
        __syncthreads();
        // (B) lambda_{n-1} of plane o = k - 2
        const int zo = k - 2;
        if (zo >= z0 && zo < z0 + ZB && zo < nz && col) {
            const int m = mrow[0];
            const T* Mo = mb + (mslot == 0 ? 2 : mslot - 1) * 6 * R::NM;   // plane k - 2
            const T* Mm = mb + (mslot == 0 ? 1 : (mslot == 1 ? 2 : 0)) * 6 * R::NM;  // plane k - 3
            const T* Mp = mk1;                                             // plane k - 1
            const long long gi = gcol + plane * zo;
            const T u[3] = {up0[0], up0[1], up0[2]};
            const T m2[3][3] = {{Mo[m], Mo[3 * R::NM + m], Mo[4 * R::NM + m]},
                                {Mo[3 * R::NM + m], Mo[R::NM + m], Mo[5 * R::NM + m]},
                                {Mo[4 * R::NM + m], Mo[5 * R::NM + m], Mo[2 * R::NM + m]}};
            // sum_a [M2_ab(z - e_a) - M2_ab(z + e_a)] for b = x, y, z
            T dA[3];
            dA[0] = (Mo[m - 1] - Mo[m + 1]) + (Mo[3 * R::NM + m - R::MX] - Mo[3 * R::NM + m + R::MX]) +
                    (Mm[4 * R::NM + m] - Mp[4 * R::NM + m]);
            dA[1] = (Mo[3 * R::NM + m - 1] - Mo[3 * R::NM + m + 1]) + (Mo[R::NM + m - R::MX] - Mo[R::NM + m + R::MX]) +
                    (Mm[5 * R::NM + m] - Mp[5 * R::NM + m]);
            dA[2] = (Mo[4 * R::NM + m - 1] - Mo[4 * R::NM + m + 1]) +
                    (Mo[5 * R::NM + m - R::MX] - Mo[5 * R::NM + m + R::MX]) + (Mm[2 * R::NM + m] - Mp[2 * R::NM + m]);
            const bool wz = !g.periodic[2] && (zo == 0 || zo == nz - 1);
            const bool wall = wall_xy || wz;
            const bool probe = a.src && !wall && probe_xy && zo >= g.probe_lo[2] && zo < g.probe_hi[2];
            a.lam_out[gi] = (T)3 * M0o;
            const T M1[3] = {M1o0, M1o1, M1o2};
            T v[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                v[e] = (T)3 * M1[e] - (T)3 * u[e] * M0o + A * dA[e];
#pragma unroll
                for (int c = 0; c < 3; ++c) v[e] += (T)9 * m2[c][e] * u[c];
            }
            if (probe) {
                const T f = src_factor(a, a.dir[0] * u[0] + a.dir[1] * u[1] + a.dir[2] * u[2]);
#pragma unroll
                for (int e = 0; e < 3; ++e) v[e] += a.phi_dir[e] * f;
            }
#pragma unroll
            for (int e = 0; e < 3; ++e) a.lam_out[(1 + e) * N + gi] = v[e];
            const int bz = colbox ? box_coord(zo, xs2, g.Fb[2], g.n[2], g.periodic[2]) : -1;
            if (bz >= 0) {
                const long long bl = bx + (long long)g.Fb[0] * (by + (long long)g.Fb[1] * bz);
#pragma unroll
                for (int c = 0; c < 3; ++c) a.boxbuf[(3 + c) * g.Fbn + bl] = uc0[c];
            }
        }
        // prefetch u_{n-1} (and u_n on the footprint box) of the next output plane
        if (col && zo + 1 >= z0 && zo + 1 < z0 + ZB && zo + 1 < nz) {
            const long long gn = gcol + plane * (zo + 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) up0[c] = a.u_prev[c * N + gn];
            if (colbox && box_coord(zo + 1, xs2, g.Fb[2], g.n[2], g.periodic[2]) >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) uc0[c] = a.u_cur[c * N + gn];
            }
        }
        T* t = sk;
        sk = sn;
        sn = t;
        mslot = mslot == 2 ? 0 : mslot + 1;
        __syncthreads();
    }
}

}  // namespace lks
