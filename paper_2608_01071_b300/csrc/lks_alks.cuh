// The paper's continuous adjoint, the ALKS (Sec. 2.5, Eqs. ap_tmp-as), as an alternative to the exact discrete
// adjoint of the forward step (lks_step_kernels.cuh).
//
// The ALKS carries the adjoint moments (p~, u~, s~) of the equilibrium's pressure, velocity and velocity-gradient
// terms; s~ is symmetric, so a state holds 1 + D + D (D + 1) / 2 fields: p~, u~_0 .. u~_D-1, then s~ in the packed
// order of sym<D>.  One reverse step, from step n to n - 1:
//   f~eq_i(z) = p~ + c_i . Q,   Q_a = 3 (u~_a + 3 s~_ab u_b - p~ u_a) - A sum_b [s~_ab(z + e_b) - s~_ab(z - e_b)]
//               (everything at node z and step n; u the flow state of step n; the central difference of s~ + s~^T),
//   p~*, u~*, s~* at x = sum_i w_i {1, c_i, c_i c_i} f~eq_i(x + c_i)                              (Eqs. ap_tmp-as_tmp)
//   p~ = p~*, s~ = s~*, u~ = (u~* - phi / 3) / (1 + kappa_{n-1}) off the walls (phi = n / (Nt |O|) on the probe
//   nodes: the objective's source, whose p~ and s~ moments vanish by symmetry; the explicit Brinkman source
//   -3 kappa c . u~ of Eq. au makes u~ implicit), 0 on walls; at n - 1 = 0 the sources are not added.
// The terminal state (step Nt) is the source alone: p~ = s~ = 0, u~ = -phi / (3 (1 + kappa_Nt)).
// The local sensitivities of step n are the ALKS forms kappa-bar = 3 (u_n - u^S_n) . u~_n and u^S-bar = -3 kappa_n
// u~_n (adj_sens_kernel with ALKS set), through the same transposed mapping as the exact adjoint.  The step kernel
// records u~_n and u_n on the footprint box of step n for them.
//
// The moment gathers are those of the exact adjoint with (p-bar*/3, u-bar*) replaced by (p~, Q), so the kernel follows
// the generic shared-memory tiles of adj_step_kernel: s~ on the halo-2 region, (p~, Q) on the halo-1 region.
#pragma once

#include "lks_step_kernels.cuh"

namespace lks {

template <int D>
struct AlksState {
    static constexpr int NS = D * (D + 1) / 2;
    static constexpr int F = 1 + D + NS;  // fields of an ALKS state
};

template <typename T>
struct AlksArgs {
    const T* lam_in;     // ALKS state of step n
    T* lam_out;          // ALKS state of step n - 1
    const T* u_cur;      // u of the flow state n (component a at u_cur + a N)
    const T* kref;
    const Pose* pose_n;  // pose of step n (footprint records)
    const Pose* pose_m;  // pose of step n - 1 (kappa_{n-1} of the Brinkman source)
    T* boxbuf;           // records of step n: u~_n (D planes, 0 on walls), then u_n (D planes)
    int src;             // 1: n - 1 >= 1 (objective and Brinkman sources of step n - 1)
    T phi_dir3[3];       // n_a / (3 Nt |O|)
};

// Terminal ALKS state: p~ = s~ = 0, u~ = -phi / (3 (1 + kappa_Nt)) off the walls.
template <typename T, int D, int HW>
__global__ void alks_init_kernel(Geom g, const Pose* __restrict__ pose, const T* __restrict__ kref, T* __restrict__ lam,
                                 AlksArgs<T> a) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x[3] = {(int)(i % g.n[0]), (int)((i / g.n[0]) % g.n[1]), (int)(i / ((long long)g.n[0] * g.n[1]))};
    T uw[3];
    const bool wall = wall_node<T, D>(g, x, uw);
    const bool probe = !wall && in_probe<D>(g, x);
    T kap = 0;
    if (probe) {
        int b[3];
        bool inbox = true;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            b[c] = box_coord(x[c], pose->xs[c], g.Fb[c], g.n[c], g.periodic[c]);
            inbox = inbox && b[c] >= 0;
        }
        T C;
        if (inbox) map_node<T, D, HW, false>(g, *pose, kref, b, kap, C, nullptr, nullptr);
    }
    constexpr int F = AlksState<D>::F;
#pragma unroll
    for (int f = 0; f < F; ++f) lam[f * g.N + i] = 0;
    if (probe) {
#pragma unroll
        for (int c = 0; c < D; ++c) lam[(1 + c) * g.N + i] = -a.phi_dir3[c] / ((T)1 + kap);
    }
}

// One ALKS reverse step n -> n - 1 on TX x TY x TZ tiles (TZ = 1 in 2D).
template <typename T, int D, int HW, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ) alks_step_kernel(Geom g, AlksArgs<T> a) {
    using L = Lattice<D>;
    using TL = Tile<D, TX, TY, TZ>;
    constexpr int S = TL::S, M = TL::M, NS = AlksState<D>::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ss = reinterpret_cast<T*>(smem_raw);  // s~ (NS fields) on the halo-2 region
    T* sp = ss + NS * S;                     // p~ on the halo-1 region
    T* sq = sp + M;                          // Q (D fields) on the halo-1 region

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    pdl_wait_then_release();

    // s~ with a halo of 2
    for (int l = tid; l < S; l += TL::NT) {
        const int i = l % TL::SX, j = (l / TL::SX) % TL::SY, k = l / (TL::SX * TL::SY);
        const long long gi = wrap(x0 - 2 + i, nx) + (long long)nx * (wrap(y0 - 2 + j, ny) +
                                                                    (long long)ny * (D == 3 ? wrap(z0 - 2 + k, nz) : 0));
#pragma unroll
        for (int f = 0; f < NS; ++f) ss[f * S + l] = a.lam_in[(1 + D + f) * N + gi];
    }
    __syncthreads();

    // p~ and Q on the halo-1 region
    const T A = (T)g.A;
    constexpr int st[3] = {1, TL::SX, TL::SX * TL::SY};
    for (int l = tid; l < M; l += TL::NT) {
        const int i = l % TL::MX, j = (l / TL::MX) % TL::MY, k = l / (TL::MX * TL::MY);
        const long long gi = wrap(x0 - 1 + i, nx) + (long long)nx * (wrap(y0 - 1 + j, ny) +
                                                                    (long long)ny * (D == 3 ? wrap(z0 - 1 + k, nz) : 0));
        const int r = (i + 1) + TL::SX * ((j + 1) + TL::SY * (k + TL::KZ));
        const T pt = a.lam_in[gi];
        T u[D], ut[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            u[c] = a.u_cur[c * N + gi];
            ut[c] = a.lam_in[(1 + c) * N + gi];
        }
        sp[l] = pt;
#pragma unroll
        for (int aa = 0; aa < D; ++aa) {
            T su = 0, div = 0;
#pragma unroll
            for (int bb = 0; bb < D; ++bb) {
                const T* sab = ss + sym<D>(aa, bb) * S;
                su += sab[r] * u[bb];
                div += sab[r + st[bb]] - sab[r - st[bb]];
            }
            sq[aa * M + l] = (T)3 * (ut[aa] + (T)3 * su - pt * u[aa]) - A * div;
        }
    }
    __syncthreads();

    // moments of f~eq_i(x + c_i) = p~ + c_i . Q at the output node
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    int xg[3] = {x0 + tx, y0 + ty, (D == 3) ? z0 + tz : 0};
    const bool active = xg[0] < nx && xg[1] < ny && (D == 2 || xg[2] < nz);
    if (!active) return;
    const int mc = (tx + 1) + TL::MX * ((ty + 1) + TL::MY * (tz + TL::KZ));
    T M0 = 0, M1[D], M2[NS];
#pragma unroll
    for (int c = 0; c < D; ++c) M1[c] = 0;
#pragma unroll
    for (int f = 0; f < NS; ++f) M2[f] = 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
        int mo = mc;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int mstride = (c == 0) ? 1 : (c == 1 ? TL::MX : TL::MX * TL::MY);
            mo += L::c(q, c) * mstride;
        }
        T f = sp[mo];
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::c(q, c) != 0) f += (T)L::c(q, c) * sq[c * M + mo];
        const T wf = (T)L::w(q) * f;
        M0 += wf;
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::c(q, c) != 0) M1[c] += (T)L::c(q, c) * wf;
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int e = c; e < D; ++e) {
                const int cc = L::c(q, c) * L::c(q, e);
                if (cc != 0) M2[sym<D>(c, e)] += (T)cc * wf;
            }
    }
    const long long gi = xg[0] + (long long)nx * (xg[1] + (long long)ny * xg[2]);
    // footprint records of step n at this node: u~_n and u_n
    {
        const Pose& P = *a.pose_n;
        int b[3] = {0, 0, 0};
        bool inbox = true;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            b[c] = box_coord(xg[c], P.xs[c], g.Fb[c], g.n[c], g.periodic[c]);
            inbox = inbox && b[c] >= 0;
        }
        if (inbox) {
            const long long bl = b[0] + (long long)g.Fb[0] * (b[1] + (long long)g.Fb[1] * b[2]);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                a.boxbuf[c * g.Fbn + bl] = a.lam_in[(1 + c) * N + gi];
                a.boxbuf[(D + c) * g.Fbn + bl] = a.u_cur[c * N + gi];
            }
        }
    }
    a.lam_out[gi] = M0;
#pragma unroll
    for (int f = 0; f < NS; ++f) a.lam_out[(1 + D + f) * N + gi] = M2[f];
    T un[D];
#pragma unroll
    for (int c = 0; c < D; ++c) un[c] = M1[c];
    if (a.src) {
        T uw[3];
        const bool wall = wall_node<T, D>(g, xg, uw);
        if (wall) {
#pragma unroll
            for (int c = 0; c < D; ++c) un[c] = 0;
        } else {
            if (in_probe<D>(g, xg)) {
#pragma unroll
                for (int c = 0; c < D; ++c) un[c] -= a.phi_dir3[c];
            }
            const Pose& P = *a.pose_m;
            int b[3];
            bool inbox = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                b[c] = box_coord(xg[c], P.xs[c], g.Fb[c], g.n[c], g.periodic[c]);
                inbox = inbox && b[c] >= 0;
            }
            T kap = 0, C;
            if (inbox) map_node<T, D, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
            const T inv = (T)1 / ((T)1 + kap);
#pragma unroll
            for (int c = 0; c < D; ++c) un[c] *= inv;
        }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) a.lam_out[(1 + c) * N + gi] = un[c];
}

}  // namespace lks
