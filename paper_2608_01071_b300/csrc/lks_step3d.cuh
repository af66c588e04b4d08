// D3Q15 forward and adjoint step kernels, marching along z (2.5D).
//
// A block owns a 32 x 8 column of (x, y) nodes and a run of ZB planes in z.  Shared memory holds rings of
// three planes: the loaded state (halo 2 in x and y), and either the 15 weighted equilibrium values
// w_i f_i of every node of the halo-1 region (forward) or its 10 local adjoint moments (adjoint).  Each
// plane of the state is read from global memory once per block (prefetched into registers one plane ahead)
// instead of once per stencil tap, and the plane-invariant index arithmetic is done once per thread.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"

namespace lks {

struct Reg3 {
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int SX = TX + 4, SY = TY + 4, NS = SX * SY;  // halo-2 region of a plane
    static constexpr int MX = TX + 2, MY = TY + 2, NM = MX * MY;  // halo-1 region of a plane
    static constexpr int PER = (NS + NT - 1) / NT;                // halo-2 elements per thread
};

template <typename T>
__host__ __device__ constexpr size_t smem3d_fwd() {
    return sizeof(T) * (3 * 4 * Reg3::NS + 3 * 15 * Reg3::NM);
}
template <typename T>
__host__ __device__ constexpr size_t smem3d_adj() {
    return sizeof(T) * (3 * 4 * Reg3::NS + 3 * 10 * Reg3::NM);
}

__device__ __forceinline__ int ring3(int k) {
    const int r = k % 3;
    return r < 0 ? r + 3 : r;
}

// ------------------------------------------------------------------------------------------------
// Forward step n-1 -> n (Sec. 2.2 / 2.3), same arithmetic as fwd_step_kernel.
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int ZB>
__global__ void __launch_bounds__(Reg3::NT) fwd3d_kernel(Geom g, FwdArgs<T> a) {
    using L = Lattice<3>;
    using R = Reg3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * (R::NT / 32)];
    T* raw = reinterpret_cast<T*>(smem_raw);  // [3 slots][4 fields][NS]
    T* wf = raw + 3 * 4 * R::NS;              // [3 slots][15][NM]

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const long long plane = (long long)nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * R::TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const T A = (T)g.A;
    const Pose& P = *a.pose;

    // plane-invariant offsets of this thread's halo-2 elements
    long long off[R::PER];
#pragma unroll
    for (int e = 0; e < R::PER; ++e) {
        const int l = tid + e * R::NT;
        const int i = l % R::SX, j = l / R::SX;
        off[e] = (l < R::NS) ? (long long)wrap(x0 - 2 + i, nx) + (long long)nx * wrap(y0 - 2 + j, ny) : 0;
    }
    pdl_wait_then_release();
    T pre[R::PER][4];
    auto fetch = [&](int k) {
        const long long base = plane * wrap(k, nz);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            if (tid + e * R::NT < R::NS) {
#pragma unroll
                for (int f = 0; f < 4; ++f) pre[e][f] = a.in[f * N + base + off[e]];
            }
        }
    };
    auto store = [&](int k) {
        T* dst = raw + ring3(k) * 4 * R::NS;
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            const int l = tid + e * R::NT;
            if (l < R::NS) {
#pragma unroll
                for (int f = 0; f < 4; ++f) dst[f * R::NS + l] = pre[e][f];
            }
        }
    };
    // prologue: planes z0-2, z0-1, z0 in the ring, z0+1 in flight
    fetch(z0 - 2);
    store(z0 - 2);
    fetch(z0 - 1);
    store(z0 - 1);
    fetch(z0);
    store(z0);
    fetch(z0 + 1);
    __syncthreads();

    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    T jacc = 0, qacc = 0;
    bool unstable = false;

    for (int k = z0 - 1; k <= z0 + ZB; ++k) {
        // (A) weighted equilibrium values of plane k on the halo-1 region
        {
            const T* rc = raw + ring3(k) * 4 * R::NS;
            const T* rm = raw + ring3(k - 1) * 4 * R::NS;
            const T* rp = raw + ring3(k + 1) * 4 * R::NS;
            T* out = wf + ring3(k) * 15 * R::NM;
            for (int l = tid; l < R::NM; l += R::NT) {
                const int i = l % R::MX, j = l / R::MX;
                const int r = (i + 1) + R::SX * (j + 1);
                const T p = rc[r];
                T u[3], G[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T* f = rc + (1 + c) * R::NS;
                    u[c] = f[r];
                    G[0][c] = (T)0.5 * (f[r + 1] - f[r - 1]);
                    G[1][c] = (T)0.5 * (f[r + R::SX] - f[r - R::SX]);
                    G[2][c] = (T)0.5 * (rp[(1 + c) * R::NS + r] - rm[(1 + c) * R::NS + r]);
                }
                const T sig = (T)3 * p - (T)1.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                T Tm[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int e = c; e < 3; ++e) {
                        Tm[c][e] = (T)4.5 * u[c] * u[e] + A * (G[c][e] + G[e][c]);
                        Tm[e][c] = Tm[c][e];
                    }
#pragma unroll
                for (int q = 0; q < L::Q; ++q) {
                    T f = sig;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (L::c(q, c) != 0) f += (T)(3 * L::c(q, c)) * u[c];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int e = c; e < 3; ++e) {
                            const int cc = L::c(q, c) * L::c(q, e) * (c == e ? 1 : 2);
                            if (cc != 0) f += (T)cc * Tm[c][e];
                        }
                    out[q * R::NM + l] = (T)L::w(q) * f;
                }
            }
        }
        __syncthreads();
        // (B) output plane k - 1: gather-stream, Brinkman, walls, objective
        const int zo = k - 1;
        if (zo >= z0 && zo < z0 + ZB && zo < nz && col) {
            const int m = (tx + 1) + R::MX * (ty + 1);
            // planes zo + 1, zo, zo - 1 feed directions with c_z = -1, 0, +1
            const T* wsl[3] = {wf + ring3(zo + 1) * 15 * R::NM + m, wf + ring3(zo) * 15 * R::NM + m,
                               wf + ring3(zo - 1) * 15 * R::NM + m};
            T accp = 0, accu[3] = {0, 0, 0};
#pragma unroll
            for (int q = 0; q < L::Q; ++q) {
                const T v = wsl[1 + L::c(q, 2)][q * R::NM - L::c(q, 0) - R::MX * L::c(q, 1)];
                accp += v;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (L::c(q, c) != 0) accu[c] += (T)L::c(q, c) * v;
            }
            const T pn = accp * (T)(1.0 / 3.0);
            T un[3];
            int xyz[3] = {xg, yg, zo};
            const int bz = box_coord(zo, P.xs[2], g.Fb[2], g.n[2], g.periodic[2]);
            if (bx >= 0 && by >= 0 && bz >= 0) {
                const int b[3] = {bx, by, bz};
                T kap, C;
                map_node<T, 3, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
                const T inv = (T)1 / ((T)1 + kap);
#pragma unroll
                for (int c = 0; c < 3; ++c) un[c] = (accu[c] + kap * (pose_uG<T>(P, c) * C)) * inv;
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) un[c] = accu[c];
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
            if (!wall) {
                if (a.u_crit2 > (T)0 && !(un[0] * un[0] + un[1] * un[1] + un[2] * un[2] <= a.u_crit2)) unstable = true;
                if (in_probe<3>(g, xyz)) {
                    const T nu = a.dir[0] * un[0] + a.dir[1] * un[1] + a.dir[2] * un[2];
                    jacc += nu;
                    qacc += nu * nu;
                }
            }
        }
        // next raw plane into the slot of plane k - 1 (no longer read), prefetch the one after
        store(k + 2);
        if (k + 3 <= z0 + ZB + 1) fetch(k + 3);
        __syncthreads();
    }
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int px = (int)blockIdx.x - a.jb_lo[0], py = (int)blockIdx.y - a.jb_lo[1], pz = (int)blockIdx.z - a.jb_lo[2];
        if (px >= 0 && px < a.jb_n[0] && py >= 0 && py < a.jb_n[1] && pz >= 0 && pz < a.jb_n[2]) {
            store_probe_partials<R::NT, T>(jacc, qacc, a.jslot, a.jsq, px + a.jb_n[0] * (py + a.jb_n[1] * pz), red);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1} (same algebra as adj_step_kernel), recording lam_u and u_n on the
// footprint box.
// ------------------------------------------------------------------------------------------------
template <typename T, int HW, int ZB>
__global__ void __launch_bounds__(Reg3::NT) adj3d_kernel(Geom g, AdjArgs<T> a) {
    using L = Lattice<3>;
    using R = Reg3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* raw = reinterpret_cast<T*>(smem_raw);  // [3 slots][4][NS]: p-bar*, u-bar*
    T* mom = raw + 3 * 4 * R::NS;             // [3 slots][10][NM]: M0, M1 (3), M2 (6, packed)

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const long long plane = (long long)nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * R::TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const T A = (T)g.A;
    const Pose& P = *a.pose;

    long long off[R::PER];
    int ex[R::PER], ey[R::PER], ebx[R::PER], eby[R::PER];
#pragma unroll
    for (int e = 0; e < R::PER; ++e) {
        const int l = tid + e * R::NT;
        const int i = l % R::SX, j = l / R::SX;
        ex[e] = wrap(x0 - 2 + i, nx);
        ey[e] = wrap(y0 - 2 + j, ny);
        off[e] = (l < R::NS) ? (long long)ex[e] + (long long)nx * ey[e] : 0;
        ebx[e] = box_coord(ex[e], P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        eby[e] = box_coord(ey[e], P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    }
    pdl_wait_then_release();
    T pre[R::PER][4];
    auto fetch = [&](int k) {
        const long long base = plane * wrap(k, nz);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            if (tid + e * R::NT < R::NS) {
#pragma unroll
                for (int f = 0; f < 4; ++f) pre[e][f] = a.lam_in[f * N + base + off[e]];
            }
        }
    };
    // p-bar* = lam_p; u-bar* = lam_u / (1 + kappa), 0 on walls
    auto store = [&](int k) {
        const int kz = wrap(k, nz);
        T* dst = raw + ring3(k) * 4 * R::NS;
        const int bz = box_coord(kz, P.xs[2], g.Fb[2], g.n[2], g.periodic[2]);
#pragma unroll
        for (int e = 0; e < R::PER; ++e) {
            const int l = tid + e * R::NT;
            if (l < R::NS) {
                int xyz[3] = {ex[e], ey[e], kz};
                T uw[3];
                T fac = 1;
                if (wall_node<T, 3>(g, xyz, uw)) {
                    fac = 0;
                } else if (ebx[e] >= 0 && eby[e] >= 0 && bz >= 0) {
                    const int b[3] = {ebx[e], eby[e], bz};
                    fac = adj_inv<T, 3, HW>(g, P, a.kref, a.fac, b);
                }
                dst[l] = pre[e][0];
#pragma unroll
                for (int f = 1; f < 4; ++f) dst[f * R::NS + l] = pre[e][f] * fac;
            }
        }
    };
    fetch(z0 - 2);
    store(z0 - 2);
    fetch(z0 - 1);
    store(z0 - 1);
    fetch(z0);
    store(z0);
    fetch(z0 + 1);
    __syncthreads();

    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);

    for (int k = z0 - 1; k <= z0 + ZB; ++k) {
        // (A) local moments of plane k on the halo-1 region: F-bar_i(y) = p-bar*(y + c_i)/3 + c_i . u-bar*(y + c_i)
        {
            const T* rs[3] = {raw + ring3(k - 1) * 4 * R::NS, raw + ring3(k) * 4 * R::NS, raw + ring3(k + 1) * 4 * R::NS};
            T* out = mom + ring3(k) * 10 * R::NM;
            for (int l = tid; l < R::NM; l += R::NT) {
                const int i = l % R::MX, j = l / R::MX;
                const int r = (i + 1) + R::SX * (j + 1);
                T M0 = 0, M1[3] = {0, 0, 0}, M2[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int q = 0; q < L::Q; ++q) {
                    const T* s = rs[1 + L::c(q, 2)];
                    const int ro = r + L::c(q, 0) + R::SX * L::c(q, 1);
                    T f = s[ro] * (T)(1.0 / 3.0);
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (L::c(q, c) != 0) f += (T)L::c(q, c) * s[(1 + c) * R::NS + ro];
                    const T wfv = (T)L::w(q) * f;
                    M0 += wfv;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (L::c(q, c) != 0) M1[c] += (T)L::c(q, c) * wfv;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int e = c; e < 3; ++e)
                            if (L::c(q, c) * L::c(q, e) != 0) M2[sym<3>(c, e)] += (T)(L::c(q, c) * L::c(q, e)) * wfv;
                }
                out[l] = M0;
#pragma unroll
                for (int c = 0; c < 3; ++c) out[(1 + c) * R::NM + l] = M1[c];
#pragma unroll
                for (int c = 0; c < 6; ++c) out[(4 + c) * R::NM + l] = M2[c];
            }
        }
        __syncthreads();
        // (B) lambda_{n-1} of plane k - 1
        const int zo = k - 1;
        if (zo >= z0 && zo < z0 + ZB && zo < nz && col) {
            const int m = (tx + 1) + R::MX * (ty + 1);
            const T* Mc = mom + ring3(zo) * 10 * R::NM;
            const T* Mm = mom + ring3(zo - 1) * 10 * R::NM;
            const T* Mp = mom + ring3(zo + 1) * 10 * R::NM;
            const long long gi = xg + (long long)nx * yg + plane * zo;
            T u[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c] = a.u_prev[c * N + gi];
            const T M0 = Mc[m];
            int xyz[3] = {xg, yg, zo};
            T uw[3];
            const bool wall = wall_node<T, 3>(g, xyz, uw);
            const bool probe = a.src && !wall && in_probe<3>(g, xyz);
            const T fsrc = probe ? src_factor(a, a.dir[0] * u[0] + a.dir[1] * u[1] + a.dir[2] * u[2]) : (T)1;
            a.lam_out[gi] = (T)3 * M0;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                T v = (T)3 * Mc[(1 + e) * R::NM + m] - (T)3 * u[e] * M0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int f = (4 + sym<3>(c, e)) * R::NM;
                    v += (T)9 * Mc[f + m] * u[c];
                    if (c == 0) v += A * (Mc[f + m - 1] - Mc[f + m + 1]);
                    if (c == 1) v += A * (Mc[f + m - R::MX] - Mc[f + m + R::MX]);
                    if (c == 2) v += A * (Mm[f + m] - Mp[f + m]);
                }
                if (probe) v += a.phi_dir[e] * fsrc;
                a.lam_out[(1 + e) * N + gi] = v;
            }
            const int bz = box_coord(zo, P.xs[2], g.Fb[2], g.n[2], g.periodic[2]);
            if (bx >= 0 && by >= 0 && bz >= 0) {
                const long long bl = bx + (long long)g.Fb[0] * (by + (long long)g.Fb[1] * bz);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a.boxbuf[c * g.Fbn + bl] = wall ? (T)0 : a.lam_in[(1 + c) * N + gi];
                    a.boxbuf[(3 + c) * g.Fbn + bl] = a.u_cur[c * N + gi];
                }
            }
        }
        store(k + 2);
        if (k + 3 <= z0 + ZB + 1) fetch(k + 3);
        __syncthreads();
    }
}

}  // namespace lks
