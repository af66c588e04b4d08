// Objective J2 of Eq. objective2 (the oar) for a translating body, and its adjoint pieces (a rotating body:
// lks_oar_rot.cuh).
//
// Without rotation x^ref_j = j + o_n, so the design-grid integral sum_j kappa^ref_j u^ref_{j,b}, with u^ref_j the
// velocity mapped back onto node j (sum_x W(x - x^ref_j) u(x)), equals sum_x kappa_n(x) u_{n,b}(x): both are the sum
// over (x, j) of W(x - x^ref_j) kappa^ref_j u_b(x).  Per step n, with S_b(n) = sum_x kappa_n(x) u_{n,b}(x) and
// K = sum_j kappa^ref_j:
//   J2_n = c_L (S_x - u^G_x K) + c_D u^G_y (S_y - u^G_y K),   c_L = 1 / (Nt |D|),  c_D = w_D / (drag_span |D|),
// (F_L + w_D F_D; the torque term T of Eq. objective2 vanishes without rotation).  The partials accumulate
// S'_b = S_b - u^G_b K per node as the sum over the footprint box of kappa_n(x) (u_b(x) - u^G_b), with u_b taken as 0
// at box nodes outside the grid (wall axes): by the partition of unity the box's kappa_n sums to K, so this is the
// same number, but inside the body u is close to u^G and the difference is formed before the large sums, in every
// precision.  Its derivatives:
//   dJ2/du_{n,b}(x)   = g_b(n) kappa_n(x), with g_x = c_L and g_y = c_D u^G_y (the adjoint source of step n);
//   dJ2/dkappa_n(x)   = g_x u_{n,x}(x) + g_y u_{n,y}(x)            (added to kappa-bar, so it reaches kappa^ref
//                                                                   through the transposed mapping, and the position
//                                                                   through dkappa_n/ds_n);
//   dJ2/du^G_{n,x}    = -c_L K,   dJ2/du^G_{n,y} = c_D (S_y - 2 u^G_y K) = c_D (S'_y - u^G_y K);
//   dJ2/dkappa^ref_j  = sum_n (-c_L u^G_x - c_D (u^G_y)^2)         (through K, the same for every design node).
#pragma once

#include "lks_step_kernels.cuh"

namespace lks {

// Weights of J2 for the kernels below.
struct OarGeom {
    double cL;  // 1 / (Nt |D|): weight of sum_x kappa u_x in F_L
    double cD;  // w_D / (drag_span |D|): weight of u^G_y sum_x kappa u_y in w_D F_D
    double cT;  // w_T / (2 pi l_m |D|): weight of omega sum_j r_j x F_j in w_T T (rotating body only)
};

// Analysis node of footprint-box node bl of a pose: its box coordinates b, grid coordinates x and node index, or
// -1 outside the grid (wall axes; periodic axes fold into one period, the box being shorter than a period).
template <int D>
__device__ __forceinline__ long long oar_box_node(const Geom& g, const Pose& P, long long bl, int (&b)[3], int (&x)[3]) {
    box_unflatten<D>(g, bl, b);
    long long gi = 0, stride = 1;
    x[2] = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        int v = P.xs[c] + b[c];
        if (g.periodic[c]) {
            if (v >= g.n[c]) v -= g.n[c];
        } else if (v < 0 || v >= g.n[c]) {
            return -1;
        }
        x[c] = v;
        gi += v * stride;
        stride *= g.n[c];
    }
    return gi;
}

// Sum over the blocks of one launch (or of one blockIdx.y row of it) without a second kernel.  Thread 0 of every
// block stores the block's NV partials (part, valid in thread 0) in scratch[block][NV] and takes a ticket; the block
// that takes the last one sums all partials in a fixed order (thread t the blocks t, t + 256, ... in turn, then the
// block's fixed tree) into out[NV] and resets the ticket for the next launch.  No block waits for another.
template <int NV>
__device__ void last_block_sum(const double (&part)[NV], double* scratch, unsigned* ticket, int nblocks, double* out,
                               double* red) {
    __shared__ unsigned last;
    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) scratch[(long long)blockIdx.x * NV + c] = part[c];
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)(nblocks - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    for (int b = tid; b < nblocks; b += 256) {
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] += __ldcg(scratch + (long long)b * NV + c);
    }
    double o[NV];
    __syncthreads();  // red is reused
    block_sum<256, NV, double>(v, o, red);
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) out[c] = o[c];
        *ticket = 0u;
    }
}

// S'_x(n), S'_y(n) over the footprint box of one step into slot[2]: per-block partials of kappa_n (u_b - u^G_b) in
// a fixed order, then their sum in the last block (scratch[nblocks][2], ticket).
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) oar_partial_kernel(Geom g, const Pose* __restrict__ pose,
                                                          const T* __restrict__ kref, const T* __restrict__ st,
                                                          double* __restrict__ scratch, unsigned* __restrict__ ticket,
                                                          double* __restrict__ slot) {
    __shared__ double red[2 * 8];
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    T v[2] = {0, 0};
    if (bl < g.Fbn) {
        int b[3], x[3];
        const long long gi = oar_box_node<D>(g, *pose, bl, b, x);
        T kap, C;
        map_node<T, D, HW, false>(g, *pose, kref, b, kap, C, nullptr, nullptr);
        const T ux = gi >= 0 ? st[g.N + gi] : (T)0, uy = gi >= 0 ? st[2 * g.N + gi] : (T)0;
        v[0] = kap * (ux - pose_uG<T>(*pose, 0));
        v[1] = kap * (uy - pose_uG<T>(*pose, 1));
    }
    double out[2];
    block_sum<256, 2, T>(v, out, red);
    last_block_sum<2>(out, scratch, ticket, (int)gridDim.x, slot, red);
}

// Adjoint source of step n: lambda_u += g(n) kappa_n on the fluid nodes of the footprint (wall nodes take no part
// in the adjoint update, as u is imposed there).  Each box node is a distinct grid node, so there are no races.
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) oar_source_kernel(Geom g, OarGeom o, const Pose* __restrict__ pose,
                                                         const T* __restrict__ kref, T* __restrict__ lam) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    int b[3], x[3];
    const long long gi = oar_box_node<D>(g, *pose, bl, b, x);
    if (gi < 0) return;
    T uw[D];
    if (wall_node<T, D>(g, x, uw)) return;
    T kap, C;
    map_node<T, D, HW, false>(g, *pose, kref, b, kap, C, nullptr, nullptr);
    lam[g.N + gi] += (T)o.cL * kap;
    lam[2 * g.N + gi] += (T)(o.cD * pose->uG[1]) * kap;
}

// J2 from the per-step partials (overwrites obj[0]), the explicit u^G terms per step (guG[n][D]) and dJ2/dK
// (dK[0]).  One block; fixed reduction order.
static __global__ void oar_reduce_kernel(OarGeom og, const double* __restrict__ slot, int Nt,
                                  const Pose* __restrict__ poses, const double* __restrict__ kref64, long long nde,
                                  int D, double* __restrict__ obj, double* __restrict__ guG, double* __restrict__ dK) {
    __shared__ double red[2][32];
    __shared__ double Ksh;
    const int tid = threadIdx.x, nw = (blockDim.x + 31) / 32;
    double k = 0.0;
    for (long long j = tid; j < nde; j += blockDim.x) k += kref64[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if ((tid & 31) == 0) red[0][tid >> 5] = k;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[0][i];
        Ksh = s;
    }
    __syncthreads();
    const double K = Ksh, cL = og.cL, cD = og.cD;
    double tot = 0.0, dk = 0.0;
    for (int n = 1 + tid; n <= Nt; n += blockDim.x) {
        const double Sx = slot[2LL * n], Sy = slot[2LL * n + 1];  // S'_b = S_b - u^G_b K
        const double ux = poses[n].uG[0], uy = poses[n].uG[1];
        tot += cL * Sx + cD * uy * Sy;
        dk += -cL * ux - cD * uy * uy;
        for (int c = 0; c < D; ++c) guG[(long long)n * D + c] = c == 0 ? -cL * K : (c == 1 ? cD * (Sy - uy * K) : 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        dk += __shfl_xor_sync(0xffffffffu, dk, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = tot;
        red[1][tid >> 5] = dk;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0, t = 0.0;
        for (int i = 0; i < nw; ++i) {
            s += red[0][i];
            t += red[1][i];
        }
        obj[0] = s;
        dK[0] = t;
    }
}

// J2's part of the local sensitivities of a segment (beside adj_sens_kernel, after it in stream order): for every
// grid node of the footprint box and step s, with u_n from the box records,
//   kappa-bar += g_x u_x + g_y u_y,   and the position terms sum_x (g_x u_x + g_y u_y) dkappa_n/ds_a into
// oms[n][D] (n = n_first + s): per-block partials, summed per step in the last block of its row
// (scratch[s][gridDim.x][D], tickets[s]).
template <typename T, int D, int HW>
__global__ void __launch_bounds__(256) oar_sens_kernel(Geom g, OarGeom o, const Pose* __restrict__ poses,
                                                       const T* __restrict__ kref, const T* __restrict__ boxbuf,
                                                       long long bstride, int n_first, T* __restrict__ kbar,
                                                       double* __restrict__ scratch, unsigned* __restrict__ tickets,
                                                       double* __restrict__ oms) {
    __shared__ double red[D * 8];
    const int s = blockIdx.y;
    const Pose& P = poses[n_first + s];
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    T mv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) mv[c] = 0;
    if (bl < g.Fbn) {
        int b[3], x[3];
        if (oar_box_node<D>(g, P, bl, b, x) >= 0) {
            const T* bb = boxbuf + (long long)s * bstride;
            const T gu = (T)o.cL * bb[D * g.Fbn + bl] + (T)(o.cD * P.uG[1]) * bb[(D + 1) * g.Fbn + bl];
            if (kbar != nullptr) kbar[(long long)s * g.Fbn + bl] += gu;
            T kap, C, dk[D], dC[D];
            map_node<T, D, HW, true>(g, P, kref, b, kap, C, dk, dC);
#pragma unroll
            for (int c = 0; c < D; ++c) mv[c] = gu * dk[c];
        }
    }
    double out[D];
    block_sum<256, D, T>(mv, out, red);
    last_block_sum<D>(out, scratch + (long long)s * gridDim.x * D, tickets + s, (int)gridDim.x,
                      oms + (long long)(n_first + s) * D, red);
}

// The explicit terms into the gradients of the reverse sweep, one thread per step n >= 1:
// dJ/ds_n += oms[n], dJ/du^G_n += guG[n]; and dJ/dkappa^ref_j += dK for every design node.
static __global__ void oar_apply_kernel(int Nt, int D, const double* __restrict__ oms,
                                 const double* __restrict__ guG, double* __restrict__ g_s, double* __restrict__ g_uG,
                                 const double* __restrict__ dK, double* __restrict__ dkref, long long nde) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nde) dkref[i] += dK[0];
    if (i >= 1 && i <= Nt) {
        for (int c = 0; c < D; ++c) {
            g_s[i * D + c] += oms[i * D + c];
            g_uG[i * D + c] += guG[i * D + c];
        }
    }
}

}  // namespace lks
