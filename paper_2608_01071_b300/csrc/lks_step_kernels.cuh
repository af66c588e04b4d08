// Forward LKS step, exact discrete adjoint step, transposed mapping and per-step reductions.
//
// Data layout in HBM (structure of arrays, x fastest): a "state" is D + 1 consecutive fields of N values,
// field 0 the reduced pressure p' = p - 1/3 (the constant 1/3 streams through Eqs. p_tmp/u_tmp unchanged,
// since sum_i w_i c_i = 0), fields 1..D the velocity components.  The adjoint state lambda = dJ/d(p, u)
// uses the same layout.
//
// Both step kernels stage a (TX+4) x (TY+4) [x (TZ+4)] halo-2 tile in shared memory: the forward's
// equilibrium at x - c_i needs the velocity gradient at x - c_i (radius 2), and the adjoint's transposed
// gradient term needs M2 at z +- e_a of moments gathered from z + c_i (radius 2).
#pragma once

#include "lks_common.cuh"

namespace lks {

template <int D, int TX, int TY, int TZ>
struct Tile {
    static constexpr int SX = TX + 4, SY = TY + 4, SZ = (D == 3) ? TZ + 4 : 1;
    static constexpr int S = SX * SY * SZ;  // halo-2 region
    static constexpr int MX = TX + 2, MY = TY + 2, MZ = (D == 3) ? TZ + 2 : 1;
    static constexpr int M = MX * MY * MZ;  // halo-1 region
    static constexpr int NT = TX * TY * TZ;
    static constexpr int KZ = (D == 3) ? 1 : 0;  // z offset flag
};

template <typename T>
struct FwdArgs {
    const T* in;        // state n-1
    T* out_p;           // p' of state n
    T* out_u;           // u of state n (component a at out_u + a N)
    const T* kref;      // kappa^ref on the extended design grid
    const Pose* pose;   // pose of step n
    double* jslot;      // objective partials of step n, one per probe block (nullptr: not needed)
    double* jsq;        // their twins for (n.u)^2 (set with jslot)
    unsigned* flag;     // stability flag (bit 0)
    T* fac_out;         // 1 / (1 + kappa) of step n on the footprint box (box_fac_kernel's layout), written by the
                        // plane-pair forward for the adjoint when set; nullptr otherwise
    int jb_lo[3];       // first block touching the probe box, per axis
    int jb_n[3];        // number of blocks touching it, per axis
    T dir[3];           // objective direction n in T
    T u_crit2;          // squared stability limit in T (<= 0 disables)
};

template <typename T>
struct AdjArgs {
    const T* lam_in;    // lambda_n
    T* lam_out;         // lambda_{n-1}
    const T* u_prev;    // u_{n-1} (component a at u_prev + a N)
    const T* u_cur;     // u_n
    const T* kref;
    const Pose* pose;   // pose of step n
    T* boxbuf;          // footprint-box record of step n: lam_u (D planes, 0 on walls) then u_n (D planes)
    const T* fac;       // 1 / (1 + kappa) of step n on the footprint box (box_fac_kernel), or nullptr
    int src;            // 1: add the objective source phi (n - 1 >= 1)
    T phi_dir[3];       // objective source weight n_a / (Nt |O|) in T
    const double* src_c0;  // 1 + 2 phi E of the variance term (device, set by the objective reduction), or nullptr
    T src_c1;           // 2 phi
    T dir[3];           // objective direction n in T
};

// Factor f of the objective source dJ/du_{n-1} = phi_dir f at a probe node.  J1 = E - phi V (Eq. objective1),
// V = S2 - E^2 with S2 the space-time mean of (n.u)^2, so f = 1 + 2 phi E - 2 phi n.u_{n-1}; f = 1 for phi = 0.
template <typename T>
__device__ __forceinline__ T src_factor(const AdjArgs<T>& a, T nu) {
    return a.src_c0 == nullptr ? (T)1 : (T)(*a.src_c0) - a.src_c1 * nu;
}

// ------------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------------

// Programmatic dependent launch: wait until the previous kernel in the stream has completed and its memory
// is visible, then let the next kernel in the stream be scheduled while this one runs.  Both are no-ops
// when the kernel was launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Asynchronous global-to-shared copy of BYTES (4, 8 or 16; cp.async, completion tracked by commit groups).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Sum of NV values over the block in the state precision T (warp shuffles, then the warp partials in warp order on
// thread 0); the block total is returned in FP64, in which the callers sum over blocks.  FP64 throughput is scarce
// on this part (a few FP64 instructions per block already take a visible share of a sensitivity pass), so
// per-node and per-warp work never touches it.  Result valid on thread 0.  Fixed reduction order, so the result
// is deterministic.  red must hold NV * (NT / 32) doubles.
template <int NT, int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], double (&out)[NV], double* red) {
    constexpr int NW = (NT + 31) / 32;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    T* rt = reinterpret_cast<T*>(red);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) rt[c * NW + (tid >> 5)] = v[c];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            T s = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) s += rt[c * NW + i];
            out[c] = (double)s;
        }
    }
}

// Objective partials of one probe block (Eq. objective1): the sums of n.u and, when jsq is set (the objective has
// the variance term), of (n.u)^2 over its probe nodes, in the block's fixed reduction order.  red must hold
// 2 * (NT / 32) doubles.
template <int NT, typename T>
__device__ __forceinline__ void store_probe_partials(T sum, T sq, double* jslot, double* jsq, long long b, double* red) {
    const bool first = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z) == 0;
    if (jsq == nullptr) {
        T v[1] = {sum};
        double s[1];
        block_sum<NT, 1, T>(v, s, red);
        if (first) jslot[b] = s[0];
        return;
    }
    T v[2] = {sum, sq};
    double s[2];
    block_sum<NT, 2, T>(v, s, red);
    if (first) {
        jslot[b] = s[0];
        jsq[b] = s[1];
    }
}

// Does the tile [x0, x0 + T) of an axis of length n touch the probe interval [lo, hi)?
__device__ __host__ inline bool tile_hits_range(int x0, int T, int lo, int hi) {
    return x0 < hi && x0 + T > lo;
}

// Does the tile [x0, x0 + T) touch the footprint box [xs, xs + Fb) (mod n on periodic axes)?
__device__ __host__ inline bool tile_hits_box(int x0, int T, int n, int xs, int Fb, int periodic) {
    int len = (n - x0 < T) ? n - x0 : T;
    int b0 = x0 - xs;
    if (periodic) {
        if (b0 < 0) b0 += n;
        return b0 < Fb || b0 + len - 1 >= n;
    }
    return b0 < Fb && b0 + len - 1 >= 0;
}

// kappa, C and (optionally) their offset derivatives at a node of the footprint box (Eqs. kappa, u_s).
template <typename T, int D, int HW, bool GRAD>
__device__ __forceinline__ void map_node(const Geom& g, const Pose& P, const T* __restrict__ kref, const int* b,
                                         T& kap, T& C, T* dk, T* dC) {
    constexpr int NTAP = 2 * HW;
    T wt[D][NTAP], dwt[D][NTAP];
    int j0[D];
    T sa[D], dsa[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        j0[a] = b[a] - 2 * HW + 1;
        sa[a] = 0;
        dsa[a] = 0;
#pragma unroll
        for (int k = 0; k < NTAP; ++k) {
            const int j = j0[a] + k;
            const bool v = (j >= 0) && (j < g.nde[a]);
            wt[a][k] = v ? pose_w<T>(P, a, k) : (T)0;
            dwt[a][k] = v ? pose_dw<T>(P, a, k) : (T)0;
            sa[a] += wt[a][k];
            dsa[a] += dwt[a][k];
        }
    }
    C = sa[0];
#pragma unroll
    for (int a = 1; a < D; ++a) C *= sa[a];
    if (GRAD) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T v = dsa[a];
#pragma unroll
            for (int c2 = 0; c2 < D; ++c2)
                if (c2 != a) v *= sa[c2];
            dC[a] = v;
            dk[a] = 0;
        }
    }
    kap = 0;
    const int sx = g.nde[0], sxy = g.nde[0] * g.nde[1];  // the extended design grid holds fewer than 2^31 nodes
    if (D == 2) {
#pragma unroll
        for (int ky = 0; ky < NTAP; ++ky) {
            const int jy = j0[1] + ky;
            if (jy < 0 || jy >= g.nde[1]) continue;
#pragma unroll
            for (int kx = 0; kx < NTAP; ++kx) {
                const int jx = j0[0] + kx;
                if (jx < 0 || jx >= g.nde[0]) continue;
                const T kr = kref[jx + sx * jy];
                kap += wt[0][kx] * wt[1][ky] * kr;
                if (GRAD) {
                    dk[0] += dwt[0][kx] * wt[1][ky] * kr;
                    dk[1] += wt[0][kx] * dwt[1][ky] * kr;
                }
            }
        }
    } else {
#pragma unroll
        for (int kz = 0; kz < NTAP; ++kz) {
            const int jz = j0[D - 1] + kz;
            if (jz < 0 || jz >= g.nde[D - 1]) continue;
#pragma unroll
            for (int ky = 0; ky < NTAP; ++ky) {
                const int jy = j0[1] + ky;
                if (jy < 0 || jy >= g.nde[1]) continue;
#pragma unroll
                for (int kx = 0; kx < NTAP; ++kx) {
                    const int jx = j0[0] + kx;
                    if (jx < 0 || jx >= g.nde[0]) continue;
                    const T kr = kref[jx + sx * jy + sxy * jz];
                    const T wyz = wt[1][ky] * wt[D - 1][kz];
                    kap += wt[0][kx] * wyz * kr;
                    if (GRAD) {
                        dk[0] += dwt[0][kx] * wyz * kr;
                        dk[1] += wt[0][kx] * dwt[1][ky] * wt[D - 1][kz] * kr;
                        dk[D - 1] += wt[0][kx] * wt[1][ky] * dwt[D - 1][kz] * kr;
                    }
                }
            }
        }
    }
}

// 1 / (1 + kappa) at footprint-box coordinates b for the adjoint's u-bar* = lam_u / (1 + kappa): read from the
// step's precomputed box field when there is one, else evaluated here.
template <typename T, int D, int HW>
__device__ __forceinline__ T adj_inv(const Geom& g, const Pose& P, const T* __restrict__ kref, const T* __restrict__ fac,
                                     const int* b) {
    if (fac != nullptr) {
        long long bl = b[D - 1];
#pragma unroll
        for (int c = D - 2; c >= 0; --c) bl = bl * g.Fb[c] + b[c];
        return fac[bl];
    }
    T kap, C;
    map_node<T, D, HW, false>(g, P, kref, b, kap, C, nullptr, nullptr);
    return (T)1 / ((T)1 + kap);
}

// Box coordinates of the flat footprint-box index bl (x fastest), in 32-bit arithmetic: the box holds fewer than
// 2^31 / 6 nodes (checked at context creation).
template <int D>
__device__ __forceinline__ void box_unflatten(const Geom& g, long long bl, int* b) {
    const unsigned u = (unsigned)bl, F0 = (unsigned)g.Fb[0];
    const unsigned q = u / F0;
    b[0] = (int)(u - q * F0);
    if (D == 2) {
        b[1] = (int)q;
        b[2] = 0;
    } else {
        const unsigned F1 = (unsigned)g.Fb[1], q2 = q / F1;
        b[1] = (int)(q - q2 * F1);
        b[2] = (int)q2;
    }
}

// 1 / (1 + kappa) over the footprint box for steps n_first .. n_first + nsteps - 1 (one box field per step,
// stride Fbn): the adjoint steps of a segment read it instead of evaluating the mapping at every staged node.
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) box_fac_kernel(Geom g, const Pose* __restrict__ poses,
                                                      const T* __restrict__ kref, int n_first, T* __restrict__ fac) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    const int j = blockIdx.y;
    int b[3];
    box_unflatten<D>(g, bl, b);
    T kap, C;
    map_node<T, D, HW, false>(g, poses[n_first + j], kref, b, kap, C, nullptr, nullptr);
    fac[j * g.Fbn + bl] = (T)1 / ((T)1 + kap);
}

// Wall test of a node; on a wall node writes the imposed velocity (later axes win where planes meet).
template <typename T, int D>
__device__ __forceinline__ bool wall_node(const Geom& g, const int* x, T* uw) {
    bool wall = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (g.periodic[a]) continue;
        int side = -1;
        if (x[a] == 0) side = 0;
        else if (x[a] == g.n[a] - 1) side = 1;
        if (side >= 0) {
            wall = true;
#pragma unroll
            for (int c2 = 0; c2 < D; ++c2) uw[c2] = (T)g.wall_u[a][side][c2];
        }
    }
    return wall;
}

template <int D>
__device__ __forceinline__ bool in_probe(const Geom& g, const int* x) {
    bool in = true;
#pragma unroll
    for (int a = 0; a < D; ++a) in = in && x[a] >= g.probe_lo[a] && x[a] < g.probe_hi[a];
    return in;
}

// ------------------------------------------------------------------------------------------------
// Forward step n-1 -> n (Sec. 2.2 Eqs. f_eq, p_tmp, u_tmp, p, u; Sec. 2.3 Eqs. kappa, u_s), fused with the
// objective partial (Eq. objective1) and the stability check.
// ------------------------------------------------------------------------------------------------
template <typename T, int D, int HW, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ) fwd_step_kernel(Geom g, FwdArgs<T> a) {
    using L = Lattice<D>;
    using TL = Tile<D, TX, TY, TZ>;
    constexpr int S = TL::S, M = TL::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * ((TX * TY * TZ + 31) / 32)];
    T* sp = reinterpret_cast<T*>(smem_raw);  // p' on the halo-2 region
    T* su = sp + S;                          // u_a on the halo-2 region
    T* ms = su + D * S;                      // sigma = 3 p' - 3/2 |u|^2 on the halo-1 region
    T* mt = ms + M;                          // T_ab = 9/2 u_a u_b + A S_ab on the halo-1 region

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    pdl_wait_then_release();

    // phase 1: load p', u with a halo of 2 (periodic wrap on every axis)
    for (int l = tid; l < S; l += TL::NT) {
        const int i = l % TL::SX, j = (l / TL::SX) % TL::SY, k = l / (TL::SX * TL::SY);
        const int gx = wrap(x0 - 2 + i, nx), gy = wrap(y0 - 2 + j, ny);
        const int gz = (D == 3) ? wrap(z0 - 2 + k, nz) : 0;
        const long long gi = gx + (long long)nx * (gy + (long long)ny * gz);
        sp[l] = a.in[gi];
#pragma unroll
        for (int c = 0; c < D; ++c) su[c * S + l] = a.in[(1 + c) * N + gi];
    }
    __syncthreads();

    // phase 2: local moment fields on the halo-1 region
    const T A = (T)g.A;
    constexpr int st[3] = {1, TL::SX, TL::SX * TL::SY};
    for (int l = tid; l < M; l += TL::NT) {
        const int i = l % TL::MX, j = (l / TL::MX) % TL::MY, k = l / (TL::MX * TL::MY);
        const int r = (i + 1) + TL::SX * ((j + 1) + TL::SY * (k + TL::KZ));
        T u[D];
        T uu = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            u[c] = su[c * S + r];
            uu += u[c] * u[c];
        }
        ms[l] = (T)3 * sp[r] - (T)1.5 * uu;
        // G[c][e] = d u_e / d x_c by central differences
        T G[D][D];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int e = 0; e < D; ++e) G[c][e] = (T)0.5 * (su[e * S + r + st[c]] - su[e * S + r - st[c]]);
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int e = c; e < D; ++e) mt[sym<D>(c, e) * M + l] = (T)4.5 * u[c] * u[e] + A * (G[c][e] + G[e][c]);
    }
    __syncthreads();

    // phase 3: gather-stream p* = 1/3 sum_i f_i(x - c_i), u* = sum_i c_i f_i(x - c_i)
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    int xg[3] = {x0 + tx, y0 + ty, (D == 3) ? z0 + tz : 0};
    const bool active = xg[0] < nx && xg[1] < ny && (D == 2 || xg[2] < nz);
    const int mc = (tx + 1) + TL::MX * ((ty + 1) + TL::MY * (tz + TL::KZ));
    const int rc = (tx + 2) + TL::SX * ((ty + 2) + TL::SY * (tz + 2 * TL::KZ));
    T accp = 0, accu[D];
#pragma unroll
    for (int c = 0; c < D; ++c) accu[c] = 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
        int mo = mc, ro = rc;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int mstride = (c == 0) ? 1 : (c == 1 ? TL::MX : TL::MX * TL::MY);
            mo -= L::c(q, c) * mstride;
            ro -= L::c(q, c) * st[c];
        }
        T f = ms[mo];
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::c(q, c) != 0) f += (T)(3 * L::c(q, c)) * su[c * S + ro];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int e = c; e < D; ++e) {
                const int cc = L::c(q, c) * L::c(q, e) * (c == e ? 1 : 2);
                if (cc != 0) f += (T)cc * mt[sym<D>(c, e) * M + mo];
            }
        const T wf = (T)L::w(q) * f;
        accp += wf;
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::c(q, c) != 0) accu[c] += (T)L::c(q, c) * wf;
    }
    const T pn = accp * (T)(1.0 / 3.0);
    T un[D];
    // Brinkman (Eq. u) with kappa and u^S = u^G C mapped from the design grid at this step's pose
    const Pose& P = *a.pose;
    int b[D];
    bool inbox = active;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        b[c] = box_coord(xg[c], P.xs[c], g.Fb[c], g.n[c], g.periodic[c]);
        inbox = inbox && b[c] >= 0;
    }
    T kap = 0, C = 0, uS[D];
#pragma unroll
    for (int c = 0; c < D; ++c) uS[c] = 0;
    if (inbox) {
        if (g.rot) {  // rotating body: kappa and u^S of this step on the footprint box (rot_box_map_kernel)
            long long bl = b[D - 1];
#pragma unroll
            for (int c = D - 2; c >= 0; --c) bl = bl * g.Fb[c] + b[c];
            const T* map = (const T*)g.rotmap;
            kap = map[bl];
#pragma unroll
            for (int c = 0; c < D; ++c) uS[c] = map[(1 + c) * g.Fbn + bl];
        } else {
            map_node<T, D, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
#pragma unroll
            for (int c = 0; c < D; ++c) uS[c] = pose_uG<T>(P, c) * C;
        }
    }
    const T inv = (T)1 / ((T)1 + kap);
#pragma unroll
    for (int c = 0; c < D; ++c) un[c] = (accu[c] + kap * uS[c]) * inv;
    T uw[D];
    const bool wall = wall_node<T, D>(g, xg, uw);
    if (wall) {
#pragma unroll
        for (int c = 0; c < D; ++c) un[c] = uw[c];
    }
    if (active) {
        const long long gi = xg[0] + (long long)nx * (xg[1] + (long long)ny * xg[2]);
        a.out_p[gi] = pn;
#pragma unroll
        for (int c = 0; c < D; ++c) a.out_u[c * N + gi] = un[c];
        if (a.u_crit2 > (T)0 && !wall) {
            T uu = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) uu += un[c] * un[c];
            if (!(uu <= a.u_crit2)) atomicOr(a.flag, 1u);
        }
    }
    // objective partial of this block (deterministic: fixed reduction order)
    if (a.jslot != nullptr) {
        const int bx = (int)blockIdx.x - a.jb_lo[0], by = (int)blockIdx.y - a.jb_lo[1], bz = (int)blockIdx.z - a.jb_lo[2];
        const bool hit = bx >= 0 && bx < a.jb_n[0] && by >= 0 && by < a.jb_n[1] && bz >= 0 && bz < a.jb_n[2];
        if (hit) {
            T nu = 0;
            if (active && !wall && in_probe<D>(g, xg)) {
#pragma unroll
                for (int c = 0; c < D; ++c) nu += a.dir[c] * un[c];
            }
            store_probe_partials<TL::NT, T>(nu, nu * nu, a.jslot, a.jsq, bx + a.jb_n[0] * (by + a.jb_n[1] * bz), red);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1}: the exact transpose of fwd_step_kernel (discrete form of the
// ALKS moments, Eqs. ap_tmp-as), fused with the local shape and motion sensitivities (Eqs. dJdgamma,
// dJdchi in discrete form):
//   u-bar* = lam_u / (1 + kappa) (0 on walls), p-bar* = lam_p
//   F-bar_i(y) = p-bar*(y + c_i)/3 + c_i . u-bar*(y + c_i);  M0, M1, M2 = sum_i w_i {1, c_i, c_i c_i} F-bar_i
//   lam_p' = 3 M0;  lam_u'_b = 3 M1_b + 9 (M2 u)_b - 3 u_b M0 + A sum_a [M2_ab(z - e_a) - M2_ab(z + e_a)] + phi
//   kappa-bar = lam_u . (u^S - u_n) / (1 + kappa),  u^S-bar = lam_u kappa / (1 + kappa)
// ------------------------------------------------------------------------------------------------
template <typename T, int D, int HW, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ) adj_step_kernel(Geom g, AdjArgs<T> a) {
    using L = Lattice<D>;
    using TL = Tile<D, TX, TY, TZ>;
    constexpr int NS = NSym<D>::value;
    constexpr int S = TL::S, M = TL::M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sp = reinterpret_cast<T*>(smem_raw);  // p-bar* on the halo-2 region
    T* su = sp + S;                          // u-bar* on the halo-2 region
    T* m0 = su + D * S;                      // M0 on the halo-1 region
    T* m1 = m0 + M;                          // M1_a
    T* m2 = m1 + D * M;                      // M2_ab (packed symmetric)

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long N = g.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    const Pose& P = *a.pose;
    pdl_wait_then_release();

    // phase 1: Brinkman and wall adjoint on the halo-2 region
    for (int l = tid; l < S; l += TL::NT) {
        const int i = l % TL::SX, j = (l / TL::SX) % TL::SY, k = l / (TL::SX * TL::SY);
        int xg[3] = {wrap(x0 - 2 + i, nx), wrap(y0 - 2 + j, ny), (D == 3) ? wrap(z0 - 2 + k, nz) : 0};
        const long long gi = xg[0] + (long long)nx * (xg[1] + (long long)ny * xg[2]);
        sp[l] = a.lam_in[gi];
        T uw[D];
        if (wall_node<T, D>(g, xg, uw)) {
#pragma unroll
            for (int c = 0; c < D; ++c) su[c * S + l] = 0;
        } else {
            int b[D];
            bool inbox = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                b[c] = box_coord(xg[c], P.xs[c], g.Fb[c], g.n[c], g.periodic[c]);
                inbox = inbox && b[c] >= 0;
            }
            const T inv = inbox ? adj_inv<T, D, HW>(g, P, a.kref, a.fac, b) : (T)1;
#pragma unroll
            for (int c = 0; c < D; ++c) su[c * S + l] = a.lam_in[(1 + c) * N + gi] * inv;
        }
    }
    __syncthreads();

    // phase 2: reverse stream and local moments on the halo-1 region
    constexpr int st[3] = {1, TL::SX, TL::SX * TL::SY};
    for (int l = tid; l < M; l += TL::NT) {
        const int i = l % TL::MX, j = (l / TL::MX) % TL::MY, k = l / (TL::MX * TL::MY);
        const int r = (i + 1) + TL::SX * ((j + 1) + TL::SY * (k + TL::KZ));
        T M0 = 0, M1[D], M2[NS];
#pragma unroll
        for (int c = 0; c < D; ++c) M1[c] = 0;
#pragma unroll
        for (int c = 0; c < NS; ++c) M2[c] = 0;
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
            int ro = r;
#pragma unroll
            for (int c = 0; c < D; ++c) ro += L::c(q, c) * st[c];
            T f = sp[ro] * (T)(1.0 / 3.0);
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (L::c(q, c) != 0) f += (T)L::c(q, c) * su[c * S + ro];
            const T wf = (T)L::w(q) * f;
            M0 += wf;
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (L::c(q, c) != 0) M1[c] += (T)L::c(q, c) * wf;
#pragma unroll
            for (int c = 0; c < D; ++c)
#pragma unroll
                for (int e = c; e < D; ++e)
                    if (L::c(q, c) * L::c(q, e) != 0) M2[sym<D>(c, e)] += (T)(L::c(q, c) * L::c(q, e)) * wf;
        }
        m0[l] = M0;
#pragma unroll
        for (int c = 0; c < D; ++c) m1[c * M + l] = M1[c];
#pragma unroll
        for (int c = 0; c < NS; ++c) m2[c * M + l] = M2[c];
    }
    __syncthreads();

    // phase 3: lambda_{n-1} at the interior nodes
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    int xg[3] = {x0 + tx, y0 + ty, (D == 3) ? z0 + tz : 0};
    const bool active = xg[0] < nx && xg[1] < ny && (D == 2 || xg[2] < nz);
    const int mc = (tx + 1) + TL::MX * ((ty + 1) + TL::MY * (tz + TL::KZ));
    const long long gi = active ? xg[0] + (long long)nx * (xg[1] + (long long)ny * xg[2]) : 0;
    const T A = (T)g.A;
    T uw[D];
    const bool wall = wall_node<T, D>(g, xg, uw);
    if (active) {
        T u[D];
#pragma unroll
        for (int c = 0; c < D; ++c) u[c] = a.u_prev[c * N + gi];
        const T M0 = m0[mc];
        a.lam_out[gi] = (T)3 * M0;
        const bool probe = a.src && !wall && in_probe<D>(g, xg);
        T nu = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) nu += a.dir[c] * u[c];
        const T f = probe ? src_factor(a, nu) : (T)1;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            T v = (T)3 * m1[e * M + mc] - (T)3 * u[e] * M0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int mstride = (c == 0) ? 1 : (c == 1 ? TL::MX : TL::MX * TL::MY);
                const T* m2s = m2 + sym<D>(c, e) * M;
                v += (T)9 * m2s[mc] * u[c];
                v += A * (m2s[mc - mstride] - m2s[mc + mstride]);
            }
            if (probe) v += a.phi_dir[e] * f;
            a.lam_out[(1 + e) * N + gi] = v;
        }
    }

    // record lam_u and u_n on the footprint box for the segment's sensitivity pass (adj_sens_kernel)
    int b[D];
    bool inbox = active;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        b[c] = box_coord(xg[c], P.xs[c], g.Fb[c], g.n[c], g.periodic[c]);
        inbox = inbox && b[c] >= 0;
    }
    if (inbox) {
        const long long bl = b[0] + (long long)g.Fb[0] * (b[1] + (D == 3 ? (long long)g.Fb[1] * b[D - 1] : 0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
            a.boxbuf[c * g.Fbn + bl] = wall ? (T)0 : a.lam_in[(1 + c) * N + gi];
            a.boxbuf[(D + c) * g.Fbn + bl] = a.u_cur[c * N + gi];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Local shape and motion sensitivities of a whole segment (Eqs. dJdgamma, dJdchi in discrete form), off the
// adjoint's critical path: one thread per (footprint-box node, step).
//   kappa-bar = lam_u . (u^S - u_n) / (1 + kappa),   u^S-bar = lam_u kappa / (1 + kappa)
//   dJ/ds_a  += kappa-bar dkappa/ds_a + (u^S-bar . u^G) dC/ds_a,   dJ/du^G_a += u^S-bar_a C
// kappa-bar goes to kbar[s][box node] (for design_gather_kernel; 0 at box nodes outside the grid); the motion terms
// are summed per block
// (FP32 within a warp, FP64 across warps) into mslot[s][block][2D].
// ------------------------------------------------------------------------------------------------
// With ALKS set the records hold the ALKS adjoint velocity u~ (lks_alks.cuh) and the sensitivities are its forms
// kappa-bar = 3 (u_n - u^S) . u~, u^S-bar = -3 kappa u~.
// Footprint-box nodes per thread of adj_sens_kernel (block b covers nodes 256 kSensNPT b .. 256 kSensNPT (b + 1) - 1,
// coalesced per sweep): the block's motion partials are reduced once for all of them.
constexpr int kSensNPT = 4;

template <typename T, int D, int HW, bool ALKS = false>
__global__ void __launch_bounds__(256) adj_sens_kernel(Geom g, const Pose* __restrict__ poses, const T* __restrict__ kref,
                                                       const T* __restrict__ boxbuf, long long bstride, int n_first,
                                                       T* __restrict__ kbar, double* __restrict__ mslot) {
    __shared__ double red[2 * D * 8];
    const int s = blockIdx.y;
    const Pose& P = poses[n_first + s];
    T mv[2 * D];
#pragma unroll
    for (int c = 0; c < 2 * D; ++c) mv[c] = 0;
#pragma unroll 1
    for (int k = 0; k < kSensNPT; ++k) {
        const long long bl = (blockIdx.x * (long long)kSensNPT + k) * 256 + threadIdx.x;
        if (bl >= g.Fbn) break;
        int b[3];
        box_unflatten<D>(g, bl, b);
        bool ingrid = true;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (!g.periodic[c]) {
                const int x = P.xs[c] + b[c];
                ingrid = ingrid && x >= 0 && x < g.n[c];
            }
        }
        if (!ingrid && kbar != nullptr) kbar[(long long)s * g.Fbn + bl] = 0;
        if (ingrid) {
            const T* bb = boxbuf + (long long)s * bstride;
            T kap, C, dk[D], dC[D];
            map_node<T, D, HW, true>(g, P, kref, b, kap, C, dk, dC);
            const T inv = (T)1 / ((T)1 + kap);
            T kb = 0, cbar = 0, usb[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const T lu = bb[c * g.Fbn + bl];
                const T uG = pose_uG<T>(P, c);
                if (ALKS) {
                    kb += lu * (bb[(D + c) * g.Fbn + bl] - uG * C);
                    usb[c] = (T)-3 * kap * lu;
                } else {
                    kb += lu * (uG * C - bb[(D + c) * g.Fbn + bl]);
                    usb[c] = lu * kap * inv;
                }
                cbar += usb[c] * uG;
            }
            kb *= ALKS ? (T)3 : inv;
            if (kbar != nullptr) kbar[(long long)s * g.Fbn + bl] = kb;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                mv[c] += kb * dk[c] + cbar * dC[c];
                mv[D + c] += usb[c] * C;
            }
        }
    }
    if (mslot != nullptr) {
        double out[2 * D];
        block_sum<256, 2 * D, T>(mv, out, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < 2 * D; ++c) mslot[((long long)s * gridDim.x + blockIdx.x) * 2 * D + c] = out[c];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Transposed mapping onto the design grid (Eq. dJdgamma in discrete form):
//   dJ/dkappa^ref_j += sum over the segment's steps n (fixed order) of sum_x W(x - x^ref_j(n)) kappa-bar_n(x).
// One thread per extended design node; a gather from the per-step footprint buffers, so no atomics.
// ------------------------------------------------------------------------------------------------
template <typename T, int D, int HW>
__global__ void design_gather_kernel(Geom g, const Pose* __restrict__ poses, const T* __restrict__ kbar,
                                     int n_first, int nsteps, long long kstride, double* __restrict__ dkref) {
    constexpr int NTAP = 2 * HW;
    const int nd = g.nde[0] * g.nde[1] * g.nde[2];  // fewer than 2^31 (checked at context creation)
    const int jl = blockIdx.x * blockDim.x + threadIdx.x;
    if (jl >= nd) return;
    const int j[3] = {jl % g.nde[0], (jl / g.nde[0]) % g.nde[1], jl / (g.nde[0] * g.nde[1])};
    // box coordinate of tap k along axis a, b = j + 2 HW - 1 - k, and its flat-offset term (-1: off the box); both
    // are the same at every step, only the grid test of non-periodic axes depends on the pose
    const int bst[3] = {1, g.Fb[0], g.Fb[0] * g.Fb[1]};
    int bc[D][NTAP], bo[D][NTAP];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < NTAP; ++k) {
            const int b = j[a] + 2 * HW - 1 - k;
            bc[a][k] = b;
            bo[a][k] = (b >= 0 && b < g.Fb[a]) ? b * bst[a] : -1;
        }
    // running FP64 sum in strict step order n = Nt..1 across calls, so that the segmentation of the
    // reverse sweep (full storage, sqrt or binomial checkpoints) cannot change the rounding
    double acc = dkref[jl];
    for (int s = nsteps - 1; s >= 0; --s) {
        const Pose& P = poses[n_first + s];
        const T* kb = kbar + (long long)s * kstride;
        bool ok[D][NTAP];
        T ww[D][NTAP];
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int k = 0; k < NTAP; ++k) {
                ok[a][k] = bo[a][k] >= 0 && (g.periodic[a] || (unsigned)(P.xs[a] + bc[a][k]) < (unsigned)g.n[a]);
                ww[a][k] = pose_w<T>(P, a, k);
            }
        }
        T sum = 0;
        if (D == 2) {
#pragma unroll
            for (int ky = 0; ky < NTAP; ++ky) {
                if (!ok[1][ky]) continue;
#pragma unroll
                for (int kx = 0; kx < NTAP; ++kx) {
                    if (!ok[0][kx]) continue;
                    sum += ww[0][kx] * ww[1][ky] * kb[bo[0][kx] + bo[1][ky]];
                }
            }
        } else {
#pragma unroll
            for (int kz = 0; kz < NTAP; ++kz) {
                if (!ok[D - 1][kz]) continue;
#pragma unroll
                for (int ky = 0; ky < NTAP; ++ky) {
                    if (!ok[1][ky]) continue;
#pragma unroll
                    for (int kx = 0; kx < NTAP; ++kx) {
                        if (!ok[0][kx]) continue;
                        sum += ww[0][kx] * ww[1][ky] * ww[D - 1][kz] * kb[bo[0][kx] + bo[1][ky] + bo[D - 1][kz]];
                    }
                }
            }
        }
        acc += (double)sum;
    }
    dkref[jl] = acc;
}

// First stage of the per-step motion sums: chunk ch of step s's per-block partials (blocks [nsb ch / nch,
// nsb (ch + 1) / nch)), summed in a fixed order (strided over the threads, then a pairwise tree) into
// mpart[s][ch][NV].  The per-step kernels below then sum the nch chunk partials in chunk order; spreading the FP64
// additions over nsteps x nch blocks keeps them off a single SM.
template <int NV>
__global__ void __launch_bounds__(128) motion_chunk_kernel(const double* __restrict__ mslot, int nsb, int nch,
                                                          double* __restrict__ mpart) {
    __shared__ double red[NV][128];
    const int st = blockIdx.x, ch = blockIdx.y, t = threadIdx.x;
    const long long lo = (long long)nsb * ch / nch, hi = (long long)nsb * (ch + 1) / nch;
    const double* ms = mslot + (long long)st * nsb * NV;
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (long long b = lo + t; b < hi; b += 128) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += ms[b * NV + q];
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q][t] = acc[q];
    __syncthreads();
#pragma unroll
    for (int w = 64; w > 0; w >>= 1) {
        if (t < w) {
#pragma unroll
            for (int q = 0; q < NV; ++q) red[q][t] += red[q][t + w];
        }
        __syncthreads();
    }
    if (t < NV) mpart[((long long)st * nch + ch) * NV + t] = red[t][0];
}

// Per-step motion sensitivities: the partials (the chunk sums of motion_chunk_kernel) summed in order (one warp
// per step; deterministic).
template <int D>
__global__ void motion_reduce_kernel(const double* __restrict__ mslot, int nsb, int n_first, int nsteps,
                                     double* __restrict__ gs, double* __restrict__ guG) {
    const int s = blockIdx.x;
    if (s >= nsteps) return;
    const int n = n_first + s;
    const double* ms = mslot + (long long)s * nsb * 2 * D;
    const int lane = threadIdx.x;
    double acc[2 * D];
#pragma unroll
    for (int c = 0; c < 2 * D; ++c) acc[c] = 0.0;
    for (int blk = lane; blk < nsb; blk += 32) {
#pragma unroll
        for (int c = 0; c < 2 * D; ++c) acc[c] += ms[(long long)blk * 2 * D + c];
    }
#pragma unroll
    for (int c = 0; c < 2 * D; ++c) {
        double v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[c] = v;
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            gs[(long long)n * D + c] = acc[c];
            guG[(long long)n * D + c] = acc[D + c];
        }
    }
}

// Objective (Eq. objective1 as a rectangle rule over n = 1..Nt): j_n and q_n = the sums of the probe blocks'
// partials of n.u and (n.u)^2 of step n (block order); E = phi sum_n j_n, S2 = phi sum_n q_n, V = S2 - E^2 and
// J1 = E - phi_var V.  Writes obj = {J1, E, V, 1 + 2 phi_var E} (the last is the adjoint source's constant).
// jsq_off = 0 (phi_var = 0): no squares were summed, J1 = E and V is NaN.  Deterministic.
static __global__ void objective_reduce_kernel(const double* __restrict__ jslot, long long jsq_off, int njb, int Nt,
                                        double phi, double phi_var, double* __restrict__ jstep,
                                        double* __restrict__ obj) {
    __shared__ double red[2][32];
    const int tid = threadIdx.x;
    double tot = 0.0, tsq = 0.0;
    for (int n = 1 + tid; n <= Nt; n += blockDim.x) {
        const double* js = jslot + (long long)n * njb;
        double v = 0.0, q = 0.0;
        for (int b = 0; b < njb; ++b) {
            v += js[b];
            if (jsq_off != 0) q += js[jsq_off + b];
        }
        jstep[n] = v;
        tot += v;
        tsq += q;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        tsq += __shfl_xor_sync(0xffffffffu, tsq, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = tot;
        red[1][tid >> 5] = tsq;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0, sq = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) {
            s += red[0][i];
            sq += red[1][i];
        }
        const double E = s * phi, V = jsq_off != 0 ? sq * phi - E * E : __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
        obj[0] = jsq_off != 0 ? E - phi_var * V : E;
        obj[1] = E;
        obj[2] = V;
        obj[3] = 1.0 + 2.0 * phi_var * E;
    }
}

}  // namespace lks
