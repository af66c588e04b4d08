// D3Q15 forward step on plane pairs with packed FP32x2 arithmetic (FP32 state only).
//
// The streamed moments of Eqs. p_tmp, u_tmp gather f_i^eq(x - c_i).  For the eight diagonal directions
// c = (sx, sy, sz) the equilibrium at a node splits into an in-plane part and a z part,
//   f^eq_c = w_c [F(sx, sy) + sz G(sx, sy)],  F = Q + 3 (sx u_x + sy u_y) + 2 sx sy T_xy,  G = 3 u_z + 2 (sx T_xz + sy T_yz)
// (Q = sigma + tr T), and for the in-plane faces f^eq_(sx,0,0) = w_f (P_x + 3 sx u_x) (P_x = sigma + T_xx), likewise
// in y.  Each node therefore evaluates, once, the value it emits to each in-plane diagonal neighbour, for the plane
// above and below (H+-(sx, sy) = w_c (F +- G), eight values) and to its four in-plane face neighbours (four values);
// a receiving node sums one value from each neighbour, with the signs of c for the momentum.  A block marches its
// columns two planes at a time: these values for planes k and k+1 are computed together, one FP32x2 instruction for
// both, and stored interleaved in shared memory as float2, so that one 8-byte shared load feeds the same stencil
// position of both planes.  Only the coupling along z between the planes of a pair and the neighbouring pairs is done
// in scalar arithmetic (a few additions per node).  Raw planes (p', u) arrive in a ring of two plane pairs; the next
// pair is fetched while the current one is being summed.  A block whose raw region lies inside the grid in x and y
// fetches each plane with one 4-D tensor copy (all four fields) issued by one thread; a block at a periodic seam
// (whose region wraps) by 16-byte asynchronous copies of every thread (4-byte copies when n_x is not a multiple of 4).
//
// Per iteration j the block holds the raw planes k-1 .. k+2 (k = z0 - 1 + 2j) and
//   (A) evaluates the emitted values of planes k, k+1 on the halo-1 region (each thread its own column and at most
//       one node of the halo-1 ring),
//   (B) sums, for its own column, the in-plane values and the emissions of planes k, k+1 to their z-neighbours, which
//       completes the moments of planes k-1 and k; Brinkman (Eqs. p, u), walls and the stores follow.
// Planes z0 - 1 .. z0 + ZB are evaluated for the ZB output planes z0 .. z0 + ZB - 1.
#pragma once

#include "lks_common.cuh"
#include "lks_step_kernels.cuh"
#include "lks_step3s.cuh"
#include "lks_tma.cuh"

namespace lks {

struct Pair3 {
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int RX = TX + 8, RY = TY + 4, RS = RX * RY;  // raw region: x0 - 4 .. x0 + TX + 3, y0 - 2 .. y0 + TY + 1
    static constexpr int MX = TX + 2, MY = TY + 2, NM = MX * MY;  // halo-1 field region
    static constexpr int NR = NM - NT;                            // halo-1 ring nodes
    static constexpr int CPR = RX / 4;                            // 16-byte chunks per raw row
    static constexpr int NCH = 4 * RY * CPR;                      // chunks of one raw plane (4 fields)
    static constexpr int PERCH = (NCH + NT - 1) / NT;
    static constexpr int NEL = 4 * RS;                            // elements of one raw plane
    static constexpr int PEREL = (NEL + NT - 1) / NT;
    static constexpr int NFLD = 12;  // float2 arrays: H+(sx, sy), H-(sx, sy) for the four (sx, sy), then E_x+, E_x-, E_y+, E_y-
    static_assert(NR <= NT, "one ring node per thread at most");
    static_assert(Sep3<TY>::MX == MX && Sep3<TY>::MY == MY, "ring_node layout");
};

__host__ __device__ constexpr size_t smem3p_fwd() {
    return sizeof(float) * 4 * 4 * Pair3::RS + sizeof(float2) * Pair3::NFLD * Pair3::NM;
}

// Prefetch the line holding p into L2 (no register is written).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// The thread that issues and waits for a block's tensor copies: the last one, in a warp without a halo-ring node
// (the ring nodes go to the first threads), so that the copy duty does not fall on a warp that already does more.
constexpr int kTmaThread = 255;
static_assert(Pair3::NT == 256, "kTmaThread is the last thread of a plane-pair block");

// Packed FP32x2 arithmetic (one instruction for both planes; rounding as the scalar instructions; a - b = fma(b, -1, a)).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 16-byte asynchronous global-to-shared copy, cached in L2 only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

// Mapped kappa and C of Eqs. kappa and u_s along one analysis column of the footprint box, for the hat kernel.
// The 2 x 2 x 2 design taps of a node factor into x, y and z weights.  The x-y part of design plane jz,
//   K_xy(jz) = sum_{kx, ky} w_x[kx] w_y[ky] kappa^ref[jx0 + kx, jy0 + ky, jz],
// is the same for every node of the column, and consecutive nodes share one of their two design planes: a window of
// two K_xy values rolls upward, and each new plane adds one (four loads) instead of evaluating all eight taps.
// Every operation is an explicitly rounded intrinsic, so that the forward step and box_fac_kernel, which both use
// this map, give kappa (and 1 / (1 + kappa)) bit for bit alike whatever the compiler contracts around them.
struct ColumnMapHat {
    float wxy[4];  // products of the valid x and y tap weights (0 for a tap outside the design grid)
    int off[4];    // design-grid offsets of the x-y taps (clamped into the grid where the weight is 0)
    float cxy;     // sum of the valid x weights times the sum of the valid y weights
    float wz[2];   // z tap weights of the step
    float win[2];  // K_xy of design planes jz0, jz0 + 1
    int jz0;       // first design plane of the window (-2^30: empty)

    __device__ __forceinline__ void init(const Geom& g, const Pose& P, int bx, int by) {
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
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                wxy[k + 2 * l] = __fmul_rn(wx[k], wy[l]);
                off[k + 2 * l] = ix[k] + g.nde[0] * iy[l];
            }
        cxy = __fmul_rn(sx, sy);
        wz[0] = P.wf[2][0];
        wz[1] = P.wf[2][1];
        jz0 = -(1 << 30);
    }
    __device__ __forceinline__ float kxy(const Geom& g, const float* __restrict__ kref, int jz) const {
        if (jz < 0 || jz >= g.nde[2]) return 0.f;
        const float* kp = kref + g.nde[0] * g.nde[1] * jz;
        float s = __fmul_rn(wxy[0], kp[off[0]]);
#pragma unroll
        for (int t = 1; t < 4; ++t) s = __fmaf_rn(wxy[t], kp[off[t]], s);
        return s;
    }
    // kappa and C at box coordinate bz of the column
    __device__ __forceinline__ void at(const Geom& g, const float* __restrict__ kref, int bz, float& kap, float& C) {
        const int j0 = bz - 1;
        if (j0 == jz0 + 1) {
            win[0] = win[1];
            win[1] = kxy(g, kref, j0 + 1);
        } else if (j0 != jz0) {
            win[0] = kxy(g, kref, j0);
            win[1] = kxy(g, kref, j0 + 1);
        }
        jz0 = j0;
        const bool v0 = j0 >= 0 && j0 < g.nde[2], v1 = j0 + 1 >= 0 && j0 + 1 < g.nde[2];
        const float wz0 = v0 ? wz[0] : 0.f, wz1 = v1 ? wz[1] : 0.f;
        kap = __fmaf_rn(wz1, win[1], __fmul_rn(wz0, win[0]));
        C = __fmul_rn(cxy, __fadd_rn(wz0, wz1));
    }
};

// 1 / (1 + kappa) over the footprint box for steps n_first .. n_first + nsteps - 1 (box_fac_kernel) for the FP32
// state and the hat kernel in 3D, with the column map of the plane-pair forward, which writes the same factors for
// the steps it recomputes: both give the same bits.
static __global__ void __launch_bounds__(256) box_fac_hat3_kernel(Geom g, const Pose* __restrict__ poses,
                                                                  const float* __restrict__ kref, int n_first,
                                                                  float* __restrict__ fac) {
    const long long bl = blockIdx.x * 256LL + threadIdx.x;
    if (bl >= g.Fbn) return;
    const int j = blockIdx.y;
    int b[3];
    box_unflatten<3>(g, bl, b);
    ColumnMapHat cm;
    cm.init(g, poses[n_first + j], b[0], b[1]);
    float kap, C;
    cm.at(g, kref, b[2], kap, C);
    fac[j * g.Fbn + bl] = __fdiv_rn(1.f, __fadd_rn(1.f, kap));
}

// Local shape and motion sensitivities of a segment (adj_sens_kernel's quantities, Eqs. dJdgamma, dJdchi in discrete
// form) for the FP32 state and the hat kernel in 3D: one thread per (footprint-box column, chunk of kSensHatZC
// planes, step) marching up its chunk of the column.  The mapping and its offset derivatives factor like the column map: per design plane jz the x-y sums
//   K(jz) = sum w_x w_y kappa^ref,   X(jz) = sum w'_x w_y kappa^ref,   Y(jz) = sum w_x w'_y kappa^ref
// (four loads serve all three; w' = dw/d offset), and at box plane bz, whose z taps are jz = bz - 1 and bz,
//   kappa = sum w_z K,   dkappa/ds = (sum w_z X, sum w_z Y, sum w'_z K),
//   C = S_x S_y S_z,   dC/ds = (S'_x S_y S_z, S_x S'_y S_z, S_x S_y S'_z)
// with S, S' the sums of the valid weights and of their derivatives (taps off the design grid have weight 0).  A
// thread sums its motion partials over its chunk and the block over its threads in FP32, in a fixed order, as
// adj_sens_kernel does (FP64 from the block sums on: the FP64 pipe of this part is narrow); blocks: the column blocks
// of the first chunk, then of the next...  kappa-bar goes to kbar as in adj_sens_kernel (0 outside the grid).
constexpr int kSensHatNT = 128, kSensHatZC = 16;

static __global__ void __launch_bounds__(kSensHatNT, 5)
    adj_sens_hat3_kernel(Geom g, const Pose* __restrict__ poses, const float* __restrict__ kref,
                         const float* __restrict__ boxbuf, long long bstride, int n_first, float* __restrict__ kbar,
                         double* __restrict__ mslot) {
    __shared__ double red[6 * (kSensHatNT / 32)];
    const int s = blockIdx.y;
    const Pose& P = poses[n_first + s];
    const int fb0 = g.Fb[0], fbxy = g.Fb[0] * g.Fb[1];
    const long long Fbn = g.Fbn;
    const int ncb = (fbxy + kSensHatNT - 1) / kSensHatNT;  // column blocks per chunk
    const int col = (blockIdx.x % ncb) * kSensHatNT + threadIdx.x;
    const int bz0 = (blockIdx.x / ncb) * kSensHatZC, bz1 = min(bz0 + kSensHatZC, g.Fb[2]);
    float mv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool colin = col < fbxy;
    bool ok = colin;
    const int bx = ok ? col % fb0 : 0, by = ok ? col / fb0 : 0;
    // box nodes outside the grid (non-periodic axes) contribute nothing and get kappa-bar = 0
    if (ok && !g.periodic[0]) ok = (unsigned)(P.xs[0] + bx) < (unsigned)g.n[0];
    if (ok && !g.periodic[1]) ok = (unsigned)(P.xs[1] + by) < (unsigned)g.n[1];
    float* kbo = colin && kbar != nullptr ? kbar + (long long)s * Fbn + col : nullptr;
    if (!ok && kbo != nullptr) {
        for (int bz = bz0; bz < bz1; ++bz) kbo[(long long)fbxy * bz] = 0.f;
    }
    if (ok) {
        float wx[2], dwx[2], wy[2], dwy[2], sx = 0.f, dsx = 0.f, sy = 0.f, dsy = 0.f;
        int ix[2], iy[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int jx = bx - 1 + k, jy = by - 1 + k;
            const bool vx = jx >= 0 && jx < g.nde[0], vy = jy >= 0 && jy < g.nde[1];
            wx[k] = vx ? P.wf[0][k] : 0.f;
            dwx[k] = vx ? P.dwf[0][k] : 0.f;
            wy[k] = vy ? P.wf[1][k] : 0.f;
            dwy[k] = vy ? P.dwf[1][k] : 0.f;
            ix[k] = vx ? jx : 0;
            iy[k] = vy ? jy : 0;
            sx += wx[k];
            dsx += dwx[k];
            sy += wy[k];
            dsy += dwy[k];
        }
        float wK[4], wX[4], wY[4];
        int off[4];
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                wK[k + 2 * l] = wx[k] * wy[l];
                wX[k + 2 * l] = dwx[k] * wy[l];
                wY[k + 2 * l] = wx[k] * dwy[l];
                off[k + 2 * l] = ix[k] + g.nde[0] * iy[l];
            }
        const float wz[2] = {P.wf[2][0], P.wf[2][1]}, dwz[2] = {P.dwf[2][0], P.dwf[2][1]};
        const float uG[3] = {P.uGf[0], P.uGf[1], P.uGf[2]};
        const int nde2 = g.nde[2], sxy = g.nde[0] * g.nde[1], xs2 = P.xs[2], nz = g.n[2];
        const bool zper = g.periodic[2] != 0;
        const float* rec = boxbuf + (long long)s * bstride + col;
        // the four x-y taps of design plane jz (0 off the design grid), and their x-y sums
        auto taps = [&](int jz, float (&kr)[4]) {
            const bool v = jz >= 0 && jz < nde2;
            const float* kp = kref + sxy * (v ? jz : 0);
#pragma unroll
            for (int t = 0; t < 4; ++t) kr[t] = v ? kp[off[t]] : 0.f;
        };
        auto xy_sums = [&](const float (&kr)[4], float& K, float& X, float& Y) {
            K = X = Y = 0.f;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                K += wK[t] * kr[t];
                X += wX[t] * kr[t];
                Y += wY[t] * kr[t];
            }
        };
        float K0, X0, Y0;  // x-y sums of design plane bz - 1
        {
            float kr[4];
            taps(bz0 - 1, kr);
            xy_sums(kr, K0, X0, Y0);
        }
        // four planes at a time: all their loads (design taps, records) are issued before any is used
        constexpr int U = 4;
#pragma unroll 1
        for (int bq = bz0; bq < bz1; bq += U) {
            float kr[U][4], rl[U][6];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int bz = bq + u;
                in[u] = bz < bz1 && (zper || (unsigned)(xs2 + bz) < (unsigned)nz);
                taps(bz < bz1 ? bz : -1, kr[u]);
                const long long o = (long long)fbxy * (in[u] ? bz : 0);
#pragma unroll
                for (int c = 0; c < 6; ++c) rl[u][c] = in[u] ? rec[c * Fbn + o] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int bz = bq + u;
                float K1, X1, Y1;  // design plane bz
                xy_sums(kr[u], K1, X1, Y1);
                if (in[u]) {
                    const bool v0 = bz >= 1, v1 = bz < nde2;  // z taps jz = bz - 1, bz on the design grid
                    const float wz0 = v0 ? wz[0] : 0.f, wz1 = v1 ? wz[1] : 0.f;
                    const float dz0 = v0 ? dwz[0] : 0.f, dz1 = v1 ? dwz[1] : 0.f;
                    const float kap = wz0 * K0 + wz1 * K1;
                    const float dk[3] = {wz0 * X0 + wz1 * X1, wz0 * Y0 + wz1 * Y1, dz0 * K0 + dz1 * K1};
                    const float sz = wz0 + wz1, dsz = dz0 + dz1;
                    const float C = sx * sy * sz;
                    const float dC[3] = {dsx * sy * sz, sx * dsy * sz, sx * sy * dsz};
                    const float inv = 1.f / (1.f + kap);
                    float kb = 0.f, cbar = 0.f, usb[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float lu = rl[u][c];
                        kb += lu * (uG[c] * C - rl[u][3 + c]);
                        usb[c] = lu * kap * inv;
                        cbar += usb[c] * uG[c];
                    }
                    kb *= inv;
                    if (kbo != nullptr) kbo[(long long)fbxy * bz] = kb;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mv[c] += kb * dk[c] + cbar * dC[c];
                        mv[3 + c] += usb[c] * C;
                    }
                } else if (bz < bz1 && kbo != nullptr) {
                    kbo[(long long)fbxy * bz] = 0.f;
                }
                K0 = K1;
                X0 = X1;
                Y0 = Y1;
            }
        }
    }
    if (mslot != nullptr) {
        double out[6];
        block_sum<kSensHatNT, 6, float>(mv, out, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) mslot[((long long)s * gridDim.x + blockIdx.x) * 6 + c] = out[c];
        }
    }
}

// Transposed mapping onto the design grid (design_gather_kernel, Eq. dJdgamma in discrete form) for the FP32 state
// and the hat kernel in 3D.  kappa-bar is 0 at footprint-box nodes outside the grid (both sensitivity kernels write
// it so), so a tap needs no grid test, only to lie in the box: its validity and offset are fixed per design node.
// The eight tap-weight products of each step are formed once per block in shared memory; a thread sums its eight
// taps per step and adds the step's sum to its FP64 running sum in strict step order n = Nt..1 (across calls too).
constexpr int kGatherHatNT = 128, kGatherHatSC = 64;  // threads per block; steps whose weights are staged at once

static __global__ void __launch_bounds__(kGatherHatNT)
    design_gather_hat3_kernel(Geom g, const Pose* __restrict__ poses, const float* __restrict__ kbar, int n_first,
                              int nsteps, long long kstride, double* __restrict__ dkref) {
    __shared__ float wp[kGatherHatSC][8];
    const int nd = g.nde[0] * g.nde[1] * g.nde[2];  // fewer than 2^31 (checked at context creation)
    const int jl = blockIdx.x * kGatherHatNT + threadIdx.x;
    const bool act = jl < nd;
    const int jx = jl % g.nde[0], jy = (jl / g.nde[0]) % g.nde[1], jz = jl / (g.nde[0] * g.nde[1]);
    // tap t = kx + 2 ky + 4 kz reads box node (j + 1 - k) per axis
    int off[8];
    bool val[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int bx = jx + 1 - (t & 1), by = jy + 1 - ((t >> 1) & 1), bz = jz + 1 - (t >> 2);
        val[t] = act && bx >= 0 && bx < g.Fb[0] && by >= 0 && by < g.Fb[1] && bz >= 0 && bz < g.Fb[2];
        off[t] = val[t] ? bx + g.Fb[0] * (by + g.Fb[1] * bz) : 0;
    }
    double acc = act ? dkref[jl] : 0.0;
    for (int c0 = nsteps - 1; c0 >= 0; c0 -= kGatherHatSC) {
        const int cn = min(kGatherHatSC, c0 + 1);  // steps c0, c0 - 1, .., c0 - cn + 1
        __syncthreads();
        for (int i = threadIdx.x; i < cn * 8; i += kGatherHatNT) {
            const int u = i >> 3, t = i & 7;
            const Pose& P = poses[n_first + c0 - u];
            wp[u][t] = P.wf[0][t & 1] * P.wf[1][(t >> 1) & 1] * P.wf[2][t >> 2];
        }
        __syncthreads();
        if (act) {
#pragma unroll 2
            for (int u = 0; u < cn; ++u) {
                const float* kb = kbar + (long long)(c0 - u) * kstride;
                float sum = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t) sum = fmaf(wp[u][t], val[t] ? kb[off[t]] : 0.f, sum);
                acc += (double)sum;
            }
        }
    }
    if (act) dkref[jl] = acc;
}

// Forward step n-1 -> n (Sec. 2.2 / 2.3); same result as fwd_step_kernel up to the order of FP additions.
// VEC4: n_x is a multiple of 4, so raw rows move in aligned 16-byte chunks that never straddle the periodic seam.
// tm: the input state as a 4-D tensor (x, y, z, field) with a box of one raw plane (RX x RY x 1 x 4), valid when
// use_tma is set (n_x a multiple of 4).
template <int HW, int ZB, bool VEC4>
__global__ void __launch_bounds__(Pair3::NT, 3)
    fwd3p_kernel(Geom g, FwdArgs<float> a, const __grid_constant__ CUtensorMap tm, int use_tma) {
    using R = Pair3;
    static_assert(ZB % 2 == 0, "planes come in pairs");
    static_assert((4 * R::RS * sizeof(float)) % 128 == 0, "tensor copies land on 128-byte boundaries");
    constexpr int NP = ZB / 2 + 1;  // iterations (field-plane pairs)
    extern __shared__ __align__(128) unsigned char smem_pair[];
    __shared__ double red[2 * (R::NT / 32)];
    __shared__ PairTma pt;
    float* raw = reinterpret_cast<float*>(smem_pair);                     // [4 planes][p', u_x, u_y, u_z][RS]
    float2* fld = reinterpret_cast<float2*>(raw + 4 * 4 * R::RS);         // [NFLD][NM]
    // emitted values: hp[s] = H+ and hm[s] = H- for (sx, sy) = (+,+), (-,+), (+,-), (-,-) (s = 0 .. 3), i.e. for the
    // receivers at (x + 1, y + 1), (x - 1, y + 1), (x + 1, y - 1), (x - 1, y - 1); ex[0] = E_x+ (receiver x + 1),
    // ex[1] = E_x- (receiver x - 1), ey likewise in y
    float2* hp = fld;
    float2* hm = fld + 4 * R::NM;
    float2* ex = fld + 8 * R::NM;
    float2* ey = fld + 10 * R::NM;

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int N = (int)g.N;  // 32-bit indexing: these kernels run only when 4 N < 2^31
    const int plane = nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * R::TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const float A = (float)g.A;
    const Pose& P = *a.pose;
    // tensor copies for a raw region inside the grid (x0 - 4 .. x0 + TX + 3, y0 - 2 .. y0 + TY + 1); x0 - 4 is a
    // multiple of 4 elements (16 bytes)
    // (and a 128-byte aligned ring, which the declaration asks for)
    const bool tma = VEC4 && use_tma != 0 && x0 >= 4 && x0 + R::TX + 4 <= nx && y0 >= 2 && y0 + R::TY + 2 <= ny &&
                     (smem_addr(raw) & 127u) == 0u;

    // plane-invariant copy descriptors of this thread's 16-byte chunks
    int goff[VEC4 ? R::PERCH : 1];
    int soff[VEC4 ? R::PERCH : 1];
    if (VEC4 && !tma) {
#pragma unroll
        for (int q = 0; q < R::PERCH; ++q) {
            const int e = tid + q * R::NT;
            soff[q] = -1;
            goff[q] = 0;
            if (e < R::NCH) {
                const int f = e / (R::RY * R::CPR), rem = e % (R::RY * R::CPR);
                const int row = rem / R::CPR, cx = rem % R::CPR;
                const int xw = wrap(x0 - 4 + 4 * cx, nx), yw = wrap(y0 - 2 + row, ny);
                goff[q] = f * N + yw * nx + xw;
                soff[q] = f * R::RS + row * R::RX + 4 * cx;
            }
        }
    }
    // raw plane k goes to ring slot (k - z0 + 2) mod 4
    auto slot = [&](int k) -> float* { return raw + ((k - z0 + 2) & 3) * 4 * R::RS; };
    auto issue = [&](int k) {
        float* dst = slot(k);
        const float* src = a.in + plane * wrap(k, nz);
        if (VEC4) {
#pragma unroll
            for (int q = 0; q < R::PERCH; ++q)
                if (soff[q] >= 0) cp_async16(dst + soff[q], src + goff[q]);
        } else {
#pragma unroll 1
            for (int e = tid; e < R::NEL; e += R::NT) {
                const int f = e / R::RS, rem = e % R::RS, row = rem / R::RX, col = rem % R::RX;
                const int go = f * N + wrap(y0 - 2 + row, ny) * nx + wrap(x0 - 4 + col, nx);
                cp_async<4>(dst + e, src + go);
            }
        }
    };
    auto issue_pair = [&](int j) {  // raw planes z0 - 2 + 2j, z0 - 1 + 2j as one copy group (one barrier phase)
        if (tma) {
            if (tid == kTmaThread) {
                uint64_t* b = &pt.bar[j & 1];
                mbar_expect_tx(b, 2 * 4 * R::RS * sizeof(float));
                tma_load_4d(slot(z0 - 2 + 2 * j), &tm, x0 - 4, y0 - 2, wrap(z0 - 2 + 2 * j, nz), 0, b);
                tma_load_4d(slot(z0 - 1 + 2 * j), &tm, x0 - 4, y0 - 2, wrap(z0 - 1 + 2 * j, nz), 0, b);
            }
        } else {
            issue(z0 - 2 + 2 * j);
            issue(z0 - 1 + 2 * j);
            cp_async_commit();
        }
    };

    // field nodes of this thread: 0 = own column, 1 = a node of the halo-1 ring (tid < NR)
    const bool has1 = tid < R::NR;
    int fi[2], fj[2];
    fi[0] = tx + 1;
    fj[0] = ty + 1;
    ring_node<R::TY>(has1 ? tid : 0, fi[1], fj[1]);
    int mrow[2], rrow[2];  // index in the halo-1 field region and in the raw region
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        mrow[s] = fi[s] + R::MX * fj[s];
        rrow[s] = (fi[s] + 3) + R::RX * (fj[s] + 1);
    }
    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    const bool colbox = col && bx >= 0 && by >= 0;
    const int xs2 = P.xs[2];
    const float uG0 = P.uGf[0], uG1 = P.uGf[1], uG2 = P.uGf[2];
    const float2 c3 = f2s(3.f), c9 = f2s(9.f), cA = f2s(A), c45 = f2s(4.5f), cm15 = f2s(-1.5f);
    const float2 w0 = f2s(2.f / 9.f), wf = f2s(1.f / 9.f), wc = f2s(1.f / 72.f);

    if (tma && tid == kTmaThread) {
        pt.init();
        tma_prefetch_map(&tm);
    }
    pdl_wait_then_release();
    issue_pair(0);
    issue_pair(1);

    // moments carried between iterations: plane k-1 without its emission from plane k (accA), and the emission of
    // plane k (the previous pair's second plane) to plane k+1 (dnB); components p*, u*_x, u*_y, u*_z
    float accA[4] = {0.f, 0.f, 0.f, 0.f}, dnB[4] = {0.f, 0.f, 0.f, 0.f};
    bool unstable = false;
    // own-column values of the current pair, kept from (A) for (B): sigma, sigma + T_zz, 3 u_z
    float2 sig0 = f2s(0.f), pz0 = f2s(0.f), uz0 = f2s(0.f);

    // wall planes of the column's x and y (Sec. 2.2 reading: where wall planes meet, the later axis' velocity wins);
    // the wall velocities are read only at wall nodes
    int wxy_axis = -1, wxy_side = 0;
    if (!g.periodic[0] && (xg == 0 || xg == nx - 1)) {
        wxy_axis = 0;
        wxy_side = xg == 0 ? 0 : 1;
    }
    if (!g.periodic[1] && (yg == 0 || yg == ny - 1)) {
        wxy_axis = 1;
        wxy_side = yg == 0 ? 0 : 1;
    }
    ColumnMapHat cmap;
    if (HW == 1 && colbox) cmap.init(g, P, bx, by);
    const int gcol = xg + nx * yg;

    // kappa and C (Eqs. kappa, u_s) at box coordinate bz of the column
    auto map_at = [&](int bz, float& kap, float& C) {
        if (HW == 1) {
            cmap.at(g, a.kref, bz, kap, C);
        } else {
            const int b[3] = {bx, by, bz};
            map_node<float, 3, HW, false>(g, P, a.kref, b, kap, C, nullptr, nullptr);
        }
    };
    // Brinkman (Eqs. p, u), walls and stores of the completed output planes zo and zo + 1 (lanes x and y of the
    // moments), both among the block's planes
    auto emit2 = [&](int zo, float2 mp, float2 mx, float2 my, float2 mz) {
        if (!col) return;
        const float2 pn = f2mul(f2s(1.f / 3.f), mp);
        float2 un[3] = {mx, my, mz};
        if (colbox) {
            const int bz0 = box_coord(zo, xs2, g.Fb[2], g.n[2], g.periodic[2]);
            const int bz1 = box_coord(zo + 1, xs2, g.Fb[2], g.n[2], g.periodic[2]);
            if (bz0 >= 0 || bz1 >= 0) {
                float2 kap = f2s(0.f), C = f2s(0.f);
                if (bz0 >= 0) map_at(bz0, kap.x, C.x);
                if (bz1 >= 0) map_at(bz1, kap.y, C.y);
                const float2 inv = f2(__fdiv_rn(1.f, __fadd_rn(1.f, kap.x)), __fdiv_rn(1.f, __fadd_rn(1.f, kap.y)));
                if (a.fac_out != nullptr) {  // the adjoint's 1 / (1 + kappa) of this step (as box_fac_kernel)
                    const int bcol = bx + g.Fb[0] * by, fbxy = g.Fb[0] * g.Fb[1];
                    if (bz0 >= 0 && zo < nz) a.fac_out[bcol + fbxy * bz0] = inv.x;
                    if (bz1 >= 0 && zo + 1 < nz) a.fac_out[bcol + fbxy * bz1] = inv.y;
                }
                const float uG[3] = {uG0, uG1, uG2};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 nw = f2mul(f2fma(kap, f2mul(f2s(uG[c]), C), un[c]), inv);
                    un[c] = f2(bz0 >= 0 ? nw.x : un[c].x, bz1 >= 0 ? nw.y : un[c].y);
                }
            }
        }
        // wall planes (zo >= 0, so plane zo + 1 is never the lower z wall)
        const int wz0 = g.periodic[2] ? -1 : (zo == 0 ? 0 : (zo == nz - 1 ? 1 : -1));
        const int wz1 = g.periodic[2] ? -1 : (zo + 1 == nz - 1 ? 1 : -1);
        const bool wall0 = wxy_axis >= 0 || wz0 >= 0, wall1 = wxy_axis >= 0 || wz1 >= 0;
        if (wall0) {
            const int ax = wz0 >= 0 ? 2 : wxy_axis, sd = wz0 >= 0 ? wz0 : wxy_side;
#pragma unroll
            for (int c = 0; c < 3; ++c) un[c].x = (float)g.wall_u[ax][sd][c];
        }
        if (wall1) {
            const int ax = wz1 >= 0 ? 2 : wxy_axis, sd = wz1 >= 0 ? wz1 : wxy_side;
#pragma unroll
            for (int c = 0; c < 3; ++c) un[c].y = (float)g.wall_u[ax][sd][c];
        }
        const int gi = gcol + plane * zo;
        const bool v0 = zo < nz, v1 = zo + 1 < nz;
        if (v0) {
            a.out_p[gi] = pn.x;
#pragma unroll
            for (int c = 0; c < 3; ++c) a.out_u[c * N + gi] = un[c].x;
        }
        if (v1) {
            a.out_p[gi + plane] = pn.y;
#pragma unroll
            for (int c = 0; c < 3; ++c) a.out_u[c * N + gi + plane] = un[c].y;
        }
        if (a.u_crit2 > 0.f) {
            const float2 uu = f2fma(un[2], un[2], f2fma(un[1], un[1], f2mul(un[0], un[0])));
            if (v0 && !wall0 && !(uu.x <= a.u_crit2)) unstable = true;
            if (v1 && !wall1 && !(uu.y <= a.u_crit2)) unstable = true;
        }
    };

#pragma unroll 1
    for (int j = 0; j < NP; ++j) {
        // raw pair j + 1 (pair j arrived one iteration earlier; both on the first)
        if (tma) {
            if (tid == kTmaThread) pt.wait(j == 0 ? 0 : j + 1, j + 1, g);
        } else {
            cp_async_wait<0>();  // this thread's copies
        }
        __syncthreads();
        if (tma && pt.bad) return;  // a wait expired (the whole block leaves; no copy is in flight)
        const int k = z0 - 1 + 2 * j;
        const float* pm = slot(k - 1);
        const float* p0 = slot(k);
        const float* p1 = slot(k + 1);
        const float* p2 = slot(k + 2);
        // (A) emitted values of planes k, k+1 at the field nodes
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && !has1) break;
            const int r = rrow[s];
            float2 U[3], Gx[3], Gy[3], Gz[3];  // twice the central differences of u_c along x, y, z
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float* a0 = p0 + (1 + c) * R::RS;
                const float* a1 = p1 + (1 + c) * R::RS;
                const float u0 = a0[r], u1 = a1[r];
                U[c] = f2(u0, u1);
                Gx[c] = f2sub(f2(a0[r + 1], a1[r + 1]), f2(a0[r - 1], a1[r - 1]));
                Gy[c] = f2sub(f2(a0[r + R::RX], a1[r + R::RX]), f2(a0[r - R::RX], a1[r - R::RX]));
                Gz[c] = f2(u1 - pm[(1 + c) * R::RS + r], p2[(1 + c) * R::RS + r] - u0);
            }
            const float2 Pp = f2(p0[r], p1[r]);
            const float2 uu = f2fma(U[2], U[2], f2fma(U[1], U[1], f2mul(U[0], U[0])));
            const float2 sig = f2fma(c3, Pp, f2mul(cm15, uu));
            const float2 Txx = f2fma(c45, f2mul(U[0], U[0]), f2mul(cA, Gx[0]));
            const float2 Tyy = f2fma(c45, f2mul(U[1], U[1]), f2mul(cA, Gy[1]));
            const float2 Tzz = f2fma(c45, f2mul(U[2], U[2]), f2mul(cA, Gz[2]));
            // twice the off-diagonal T
            const float2 Txy2 = f2fma(c9, f2mul(U[0], U[1]), f2mul(cA, f2add(Gx[1], Gy[0])));
            const float2 Txz2 = f2fma(c9, f2mul(U[0], U[2]), f2mul(cA, f2add(Gx[2], Gz[0])));
            const float2 Tyz2 = f2fma(c9, f2mul(U[1], U[2]), f2mul(cA, f2add(Gy[2], Gz[1])));
            const float2 px = f2add(sig, Txx), py = f2add(sig, Tyy);
            const float2 Q = f2add(f2add(px, Tyy), Tzz);
            // F(sx, sy) = Q + 3 (sx u_x + sy u_y) + 2 sx sy T_xy,  G(sx, sy) = 3 u_z + 2 (sx T_xz + sy T_yz)
            const float2 t1 = f2add(Q, Txy2), t2 = f2sub(Q, Txy2);
            const float2 v1 = f2mul(c3, f2add(U[0], U[1])), v2 = f2mul(c3, f2sub(U[0], U[1]));
            const float2 uz3 = f2mul(c3, U[2]);
            const float2 g1 = f2add(Txz2, Tyz2), g2 = f2sub(Txz2, Tyz2);
            const float2 F[4] = {f2add(t1, v1), f2sub(t2, v2), f2add(t2, v2), f2sub(t1, v1)};
            const float2 G[4] = {f2add(uz3, g1), f2sub(uz3, g2), f2add(uz3, g2), f2sub(uz3, g1)};
            const int m = mrow[s];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                hp[q * R::NM + m] = f2mul(wc, f2add(F[q], G[q]));
                hm[q * R::NM + m] = f2mul(wc, f2sub(F[q], G[q]));
            }
            const float2 ux3 = f2mul(c3, U[0]), uy3 = f2mul(c3, U[1]);
            ex[m] = f2mul(wf, f2add(px, ux3));
            ex[R::NM + m] = f2mul(wf, f2sub(px, ux3));
            ey[m] = f2mul(wf, f2add(py, uy3));
            ey[R::NM + m] = f2mul(wf, f2sub(py, uy3));
            if (s == 0) {  // the own column, for (B)
                sig0 = sig;
                pz0 = f2add(sig, Tzz);
                uz0 = uz3;
            }
        }
        __syncthreads();
        // raw pair j + 2 into the slots of pair j, read for the last time in (A) above
        if (j + 2 <= NP) issue_pair(j + 2);
        // (B) sums of the emitted values at this thread's column
        {
            const int m = mrow[0];
            // receivers at (x, y) take H(+,+) from (x-1, y-1), H(-,+) from (x+1, y-1), H(+,-) from (x-1, y+1) and
            // H(-,-) from (x+1, y+1): sum, and the x and y first moments with the signs of c
            auto gather = [&](const float2* h, float2& S, float2& Dx, float2& Dy) {
                const float2 va = h[m - 1 - R::MX], vb = h[R::NM + m + 1 - R::MX], vc = h[2 * R::NM + m - 1 + R::MX],
                             vd = h[3 * R::NM + m + 1 + R::MX];
                const float2 s1 = f2add(va, vb), s2 = f2add(vc, vd);
                S = f2add(s1, s2);
                Dy = f2sub(s1, s2);
                Dx = f2add(f2sub(va, vb), f2sub(vc, vd));
            };
            float2 dnP, dnX, dnY, upP, upX, upY;
            gather(hp, dnP, dnX, dnY);
            gather(hm, upP, upX, upY);
            const float2 exm = ex[m - 1], exp_ = ex[R::NM + m + 1], eym = ey[m - R::MX], eyp = ey[R::NM + m + R::MX];
            const float2 inP = f2fma(w0, sig0, f2add(f2add(exm, exp_), f2add(eym, eyp)));
            const float2 inX = f2sub(exm, exp_), inY = f2sub(eym, eyp);
            // z faces from the column's own values
            dnP = f2add(dnP, f2mul(wf, f2add(pz0, uz0)));
            upP = f2add(upP, f2mul(wf, f2sub(pz0, uz0)));
            // plane k-1 gets the emission of plane k; plane k the one of plane k+1 (and the carried one of k-1)
            const float oA0 = accA[0] + upP.x, oA1 = accA[1] + upX.x, oA2 = accA[2] + upY.x, oA3 = accA[3] - upP.x;
            const float oB0 = (inP.x + dnB[0]) + upP.y, oB1 = (inX.x + dnB[1]) + upX.y, oB2 = (inY.x + dnB[2]) + upY.y,
                        oB3 = dnB[3] - upP.y;
            accA[0] = inP.y + dnP.x;
            accA[1] = inX.y + dnX.x;
            accA[2] = inY.y + dnY.x;
            accA[3] = dnP.x;
            dnB[0] = dnP.y;
            dnB[1] = dnX.y;
            dnB[2] = dnY.y;
            dnB[3] = dnP.y;
            if (j >= 1) emit2(k - 1, f2(oA0, oB0), f2(oA1, oB1), f2(oA2, oB2), f2(oA3, oB3));
        }
    }
    if (unstable) atomicOr(a.flag, 1u);
    if (a.jslot != nullptr) {
        const int px = (int)blockIdx.x - a.jb_lo[0], py = (int)blockIdx.y - a.jb_lo[1], pz = (int)blockIdx.z - a.jb_lo[2];
        if (px >= 0 && px < a.jb_n[0] && py >= 0 && py < a.jb_n[1] && pz >= 0 && pz < a.jb_n[2]) {
            // objective partials from this thread's own outputs, re-read after the march (planes upward)
            float jacc = 0.f, qacc = 0.f;
            if (col) {
                for (int zo = max(z0, g.probe_lo[2]); zo < min(min(z0 + ZB, nz), g.probe_hi[2]); ++zo) {
                    int xyz[3] = {xg, yg, zo};
                    float uw[3];
                    if (!in_probe<3>(g, xyz) || wall_node<float, 3>(g, xyz, uw)) continue;
                    const int gi = xg + nx * yg + plane * zo;
                    const float nu = a.dir[0] * a.out_u[gi] + a.dir[1] * a.out_u[N + gi] + a.dir[2] * a.out_u[2 * N + gi];
                    jacc += nu;
                    qacc += nu * nu;
                }
            }
            store_probe_partials<R::NT, float>(jacc, qacc, a.jslot, a.jsq, px + a.jb_n[0] * (py + a.jb_n[1] * pz), red);
        }
    }
}


// ------------------------------------------------------------------------------------------------
// Adjoint step lambda_n -> lambda_{n-1} on plane pairs (packed FP32x2); the algebra of adj3s_kernel.
//
// With P = p-bar*/3 = lambda_p/3 and (X, Y, Z) = u-bar* = lambda_u/(1 + kappa) (0 on walls) staged on the halo-2
// region as float2 pairs of planes (k, k+1), the local moments M0, M1, M2 of the planes are gathers from y + c_i that
// factor into S g = g(+1) + g(-1) and D g = g(+1) - g(-1) products over the in-plane diagonal neighbours, plus the
// face terms; a plane emits U = w (E + Z) to the plane below and L = w (E - Z) to the plane above.  A pair of raw
// planes (k, k+1) therefore completes the moments of planes k-1 and k: one completed pair C_j per iteration, whose
// M2 goes to shared memory on the halo-1 region (the A term needs its in-plane neighbours) and whose M0, M1 stay
// with the own column.  The output pair is C_{j-1}, written one iteration later, when the M2 of the plane above it
// is known: every step of the output is FP32x2 as well, with the M2 z-neighbours taken from the column itself.
//
// Iteration j: raw pair j (planes z0 - 2 + 2j, z0 - 1 + 2j) -> C_j (planes z0 - 3 + 2j, z0 - 2 + 2j);
// output C_{j-1} (planes z0 - 5 + 2j, z0 - 4 + 2j) for j >= 2.  Raw lambda arrives one pair ahead (by tensor copies
// issued by one thread where the block's raw region lies inside the grid in x and y, else by every thread's
// asynchronous copies) and is transformed into the staged pair one iteration ahead of use.
// ------------------------------------------------------------------------------------------------
struct PairA3 {
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int RX = TX + 8, RY = TY + 4, RS = RX * RY;  // raw lambda: x0 - 4 .. x0 + TX + 3, y0 - 2 .. y0 + TY + 1
    static constexpr int SX = TX + 4, SY = TY + 4, NS = SX * SY;  // staged P, X, Y, Z (halo 2): x0 - 2 .. x0 + TX + 1
    static constexpr int MX = TX + 2, MY = TY + 2, NM = MX * MY;  // moments (halo 1)
    static constexpr int NR = NM - NT;
    static constexpr int CPR = RX / 4, NCH = 4 * RY * CPR, PERCH = (NCH + NT - 1) / NT;
    static constexpr int NEL = 4 * RS;
    static constexpr int PERT = (NS + NT - 1) / NT;  // staged elements per thread
    // per moment slot: M2 xx, yy, xy, xz, yz, zz over the halo-1 region, then M0, M1x, M1y, M1z of the own columns
    static constexpr int SLOT = 6 * NM + 4 * NT;
    static_assert(NR <= NT && PERT == 2, "layout");
};

__host__ __device__ constexpr size_t smem3p_adj() {
    return sizeof(float) * 2 * 2 * 4 * PairA3::RS + sizeof(float2) * (2 * 4 * PairA3::NS + 2 * PairA3::SLOT);
}

// tm: lambda_n as a 4-D tensor (x, y, z, field) with a box of one raw plane (RX x RY x 1 x 4), valid when use_tma
// is set (n_x a multiple of 4).
template <int HW, int ZB, bool VEC4>
__global__ void __launch_bounds__(PairA3::NT, 2)
    adj3p_kernel(Geom g, AdjArgs<float> a, const __grid_constant__ CUtensorMap tm, int use_tma) {
    using R = PairA3;
    static_assert(ZB % 2 == 0, "planes come in pairs");
    static_assert((4 * R::RS * sizeof(float)) % 128 == 0, "tensor copies land on 128-byte boundaries");
    constexpr int NRP = ZB / 2 + 2;  // raw pairs
    constexpr int NJ = ZB / 2 + 3;   // iterations: raw pairs 0 .. NRP - 1, outputs of C_1 .. C_{NRP - 1}
    extern __shared__ __align__(128) unsigned char smem_pair[];
    __shared__ PairTma pt;
    float* stg = reinterpret_cast<float*>(smem_pair);                 // [2 pair slots][2 planes][4 fields][RS]
    float2* tl = reinterpret_cast<float2*>(stg + 2 * 2 * 4 * R::RS);  // [2 slots][P, X, Y, Z][NS]
    float2* mom = tl + 2 * 4 * R::NS;                                 // [2 slots][SLOT]

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int N = (int)g.N;  // 32-bit indexing: these kernels run only when 4 N < 2^31
    const int plane = nx * ny;
    const int x0 = blockIdx.x * R::TX, y0 = blockIdx.y * R::TY, z0 = blockIdx.z * ZB;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + R::TX * ty;
    const Pose& P = *a.pose;
    const int xs2 = P.xs[2];
    const bool zper = g.periodic[2] != 0;
    // tensor copies for a raw region inside the grid (x0 - 4 .. x0 + TX + 3, y0 - 2 .. y0 + TY + 1) and a 128-byte
    // aligned staging area
    const bool tma = VEC4 && use_tma != 0 && x0 >= 4 && x0 + R::TX + 4 <= nx && y0 >= 2 && y0 + R::TY + 2 <= ny &&
                     (smem_addr(stg) & 127u) == 0u;

    // raw copies: plane-invariant descriptors of this thread's 16-byte chunks
    int goff[VEC4 ? R::PERCH : 1];
    int soff[VEC4 ? R::PERCH : 1];
    if (VEC4 && !tma) {
#pragma unroll
        for (int q = 0; q < R::PERCH; ++q) {
            const int e = tid + q * R::NT;
            soff[q] = -1;
            goff[q] = 0;
            if (e < R::NCH) {
                const int f = e / (R::RY * R::CPR), rem = e % (R::RY * R::CPR);
                const int row = rem / R::CPR, cx = rem % R::CPR;
                const int xw = wrap(x0 - 4 + 4 * cx, nx), yw = wrap(y0 - 2 + row, ny);
                goff[q] = f * N + yw * nx + xw;
                soff[q] = f * R::RS + row * R::RX + 4 * cx;
            }
        }
    }
    auto issue_plane = [&](float* dst, int k) {
        const float* src = a.lam_in + plane * wrap(k, nz);
        if (VEC4) {
#pragma unroll
            for (int q = 0; q < R::PERCH; ++q)
                if (soff[q] >= 0) cp_async16(dst + soff[q], src + goff[q]);
        } else {
#pragma unroll 1
            for (int e = tid; e < R::NEL; e += R::NT) {
                const int f = e / R::RS, rem = e % R::RS, row = rem / R::RX, col = rem % R::RX;
                const int go = f * N + wrap(y0 - 2 + row, ny) * nx + wrap(x0 - 4 + col, nx);
                cp_async<4>(dst + e, src + go);
            }
        }
    };
    auto issue_pair = [&](int jj) {  // raw pair jj into staging slot jj % 2 (one barrier phase)
        float* dst = stg + (jj & 1) * 2 * 4 * R::RS;
        if (tma) {
            if (tid == kTmaThread) {
                uint64_t* b = &pt.bar[jj & 1];
                mbar_expect_tx(b, 2 * 4 * R::RS * sizeof(float));
                tma_load_4d(dst, &tm, x0 - 4, y0 - 2, wrap(z0 - 2 + 2 * jj, nz), 0, b);
                tma_load_4d(dst + 4 * R::RS, &tm, x0 - 4, y0 - 2, wrap(z0 - 1 + 2 * jj, nz), 0, b);
            }
        } else {
            issue_plane(dst, z0 - 2 + 2 * jj);
            issue_plane(dst + 4 * R::RS, z0 - 1 + 2 * jj);
            cp_async_commit();
        }
    };

    // staged elements of this thread (halo-2 region): wall and footprint coordinates, and whether the element is one
    // of the block's own columns (whose lambda_u footprint records this block writes)
    int esi[R::PERT], ebl[R::PERT];  // staging index; footprint-box offset in the x-y plane (-1: off the box)
    bool ewall[R::PERT], einner[R::PERT];
#pragma unroll
    for (int q = 0; q < R::PERT; ++q) {
        const int e = tid + q * R::NT;
        const int i = e % R::SX, jr = e / R::SX;
        const int ex = wrap(x0 - 2 + i, nx), ey = wrap(y0 - 2 + jr, ny);
        const int ebx = box_coord(ex, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
        const int eby = box_coord(ey, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
        esi[q] = (i + 2) + R::RX * jr;
        ebl[q] = (e < R::NS && ebx >= 0 && eby >= 0) ? ebx + g.Fb[0] * eby : -1;
        ewall[q] = (!g.periodic[0] && (ex == 0 || ex == nx - 1)) || (!g.periodic[1] && (ey == 0 || ey == ny - 1));
        einner[q] = e < R::NS && i >= 2 && i < R::TX + 2 && jr >= 2 && jr < R::TY + 2 && x0 - 2 + i < nx &&
                    y0 - 2 + jr < ny && ebl[q] >= 0;
    }
    const int fbxy = g.Fb[0] * g.Fb[1];
    const int Fbn = (int)g.Fbn;
    // 1 / (1 + kappa) of this thread's staged elements for the two planes of raw pair jj (1 off the footprint box,
    // 0 on walls), read one iteration ahead of the transform
    auto load_fac = [&](int jj, float (&fc)[R::PERT][2]) {
        const int q0 = z0 - 2 + 2 * jj;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kz = wrap(q0 + h, nz);
            const int bz = box_coord(kz, xs2, g.Fb[2], g.n[2], g.periodic[2]);
            const bool wz = !zper && (kz == 0 || kz == nz - 1);
            const float* fz = a.fac + fbxy * bz;
#pragma unroll
            for (int q = 0; q < R::PERT; ++q) {
                fc[q][h] = (ewall[q] || wz) ? 0.f : 1.f;
                if (!(ewall[q] || wz) && ebl[q] >= 0 && bz >= 0) fc[q][h] = fz[ebl[q]];
            }
        }
    };
    // transform raw pair jj (staging slot jj % 2) into staged slot jj % 2 with the factors fc; lambda_u records of the
    // own footprint nodes
    auto transform = [&](int jj, const float (&fc)[R::PERT][2]) {
        const float* s0 = stg + (jj & 1) * 2 * 4 * R::RS;
        const float* s1 = s0 + 4 * R::RS;
        float2* t = tl + (jj & 1) * 4 * R::NS;
        const int q0 = z0 - 2 + 2 * jj;
        int bzo[2];  // box offset of the plane, or -1 when no record is written for it
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kz = wrap(q0 + h, nz);
            const int bz = box_coord(kz, xs2, g.Fb[2], g.n[2], g.periodic[2]);
            const bool own = q0 + h >= z0 && q0 + h < z0 + ZB && q0 + h < nz;
            bzo[h] = (own && bz >= 0) ? fbxy * bz : -1;
        }
#pragma unroll
        for (int q = 0; q < R::PERT; ++q) {
            const int e = tid + q * R::NT;
            if (e >= R::NS) continue;
            const int si = esi[q];
            t[e] = f2(s0[si] * (1.f / 3.f), s1[si] * (1.f / 3.f));
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                const float l0 = s0[c * R::RS + si], l1 = s1[c * R::RS + si];
                t[c * R::NS + e] = f2(l0 * fc[q][0], l1 * fc[q][1]);
                if (einner[q]) {
                    // records of lambda_u on the box (0 on walls: the factor is 0 there)
                    if (bzo[0] >= 0) a.boxbuf[(c - 1) * Fbn + bzo[0] + ebl[q]] = fc[q][0] == 0.f ? 0.f : l0;
                    if (bzo[1] >= 0) a.boxbuf[(c - 1) * Fbn + bzo[1] + ebl[q]] = fc[q][1] == 0.f ? 0.f : l1;
                }
            }
        }
    };

    // field nodes: 0 = own column, 1 = a node of the halo-1 ring (tid < NR)
    const bool has1 = tid < R::NR;
    int fi[2], fj[2];
    fi[0] = tx + 1;
    fj[0] = ty + 1;
    ring_node<R::TY>(has1 ? tid : 0, fi[1], fj[1]);
    int mrow[2], rrow[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        mrow[s] = fi[s] + R::MX * fj[s];
        rrow[s] = (fi[s] + 1) + R::SX * (fj[s] + 1);
    }
    const int xg = x0 + tx, yg = y0 + ty;
    const bool col = xg < nx && yg < ny;
    const int gcol = xg + nx * yg;
    const int bx = box_coord(xg, P.xs[0], g.Fb[0], g.n[0], g.periodic[0]);
    const int by = box_coord(yg, P.xs[1], g.Fb[1], g.n[1], g.periodic[1]);
    const bool colbox = col && bx >= 0 && by >= 0;
    const bool probe_xy = a.src && xg >= g.probe_lo[0] && xg < g.probe_hi[0] && yg >= g.probe_lo[1] && yg < g.probe_hi[1] &&
                          !((!g.periodic[0] && (xg == 0 || xg == nx - 1)) || (!g.periodic[1] && (yg == 0 || yg == ny - 1)));
    const float2 w0 = f2s(2.f / 9.f), wf = f2s(1.f / 9.f), wc = f2s(1.f / 72.f), c3 = f2s(3.f), c9 = f2s(9.f);
    const float2 cA = f2s((float)g.A), cm3 = f2s(-3.f);

    if (tma && tid == kTmaThread) {
        pt.init();
        tma_prefetch_map(&tm);
    }
    pdl_wait_then_release();
    float fcur[R::PERT][2], fnext[R::PERT][2];
    issue_pair(0);
    load_fac(0, fcur);
    if (tma) {
        if (tid == kTmaThread) pt.wait(0, 0, g);
    } else {
        cp_async_wait<0>();
    }
    __syncthreads();
    if (tma && pt.bad) return;  // a wait expired (the whole block leaves; no copy is in flight)
    transform(0, fcur);
    issue_pair(1);
    load_fac(1, fnext);

    // From the previous pair (planes k-2, k-1): its emissions to the plane above, as pairs of the distinct terms
    // L0, L1, L2, L3, L0 + zu (own node; the ring node needs L0 .. L3), and the in-plane terms of its second plane
    // (in0, in1, in2, fx, fy; the ring node fx, fy).  z-neighbour M2 (xz, yz, zz) of the plane below the output pair.
    float2 pL0[5], pL1[4];
    float pI0[5], pI1[2];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        pL0[c] = f2s(0.f);
        pI0[c] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) pL1[c] = f2s(0.f);
    pI1[0] = pI1[1] = 0.f;
    float zm[3] = {0.f, 0.f, 0.f};

#pragma unroll 1
    for (int j = 0; j < NJ; ++j) {
        // u_{n-1} of this iteration's output pair (planes z0 - 5 + 2j, + 1), and u_n there on the footprint box (for
        // its records): prefetched into L2 here, ahead of the moments, and loaded for the output stage (no registers
        // held across the moments)
        const int o0 = z0 - 5 + 2 * j;
        bool ok[2];
        int bzo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            ok[h] = j >= 2 && col && o0 + h >= z0 && o0 + h < z0 + ZB && o0 + h < nz;
            bzo[h] = (ok[h] && colbox) ? box_coord(o0 + h, xs2, g.Fb[2], g.n[2], g.periodic[2]) : -1;
        }
        const int gi0 = gcol + plane * o0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (ok[h]) prefetch_l2(a.u_prev + gi0 + h * plane + c * N);
                if (bzo[h] >= 0) prefetch_l2(a.u_cur + gi0 + h * plane + c * N);
            }
        }
        // raw pair j + 1
        if (tma) {
            if (tid == kTmaThread && j + 1 < NRP) pt.wait(j + 1, j + 1, g);
        } else {
            cp_async_wait<0>();  // this thread's copies
        }
        __syncthreads();
        if (tma && pt.bad) return;
#pragma unroll
        for (int q = 0; q < R::PERT; ++q) {
            fcur[q][0] = fnext[q][0];
            fcur[q][1] = fnext[q][1];
        }
        if (j + 2 < NRP) {
            issue_pair(j + 2);
            load_fac(j + 2, fnext);
        }
        if (j + 1 < NRP) transform(j + 1, fcur);
        if (j < NRP) {
            // (B) moments of planes k-1, k from raw pair j = (k, k+1), k = z0 - 2 + 2j
            const float2* tP = tl + (j & 1) * 4 * R::NS;
            const float2* tX = tP + R::NS;
            const float2* tY = tP + 2 * R::NS;
            const float2* tZ = tP + 3 * R::NS;
            float2* ms = mom + (j & 1) * R::SLOT;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (s == 1 && !has1) break;
                const int r = rrow[s];
                // S/D products over the diagonal neighbours; here D g = g(+1) - g(-1)
                auto sd4 = [&](const float2* f, float2& SS, float2& DS, float2& SD, float2& DD) {
                    const float2 va = f[r - 1 - R::SX], vb = f[r + 1 - R::SX], vc = f[r - 1 + R::SX], vd = f[r + 1 + R::SX];
                    const float2 s1 = f2add(va, vb), s2 = f2add(vc, vd), d1 = f2sub(vb, va), d2 = f2sub(vd, vc);
                    SS = f2add(s1, s2);
                    SD = f2sub(s2, s1);
                    DS = f2add(d1, d2);
                    DD = f2sub(d2, d1);
                };
                float2 E0, E1, E2, E3, SS, DS, SD, DD;
                sd4(tP, SS, DS, SD, DD);
                E0 = SS;
                E1 = DS;
                E2 = SD;
                E3 = DD;
                sd4(tX, SS, DS, SD, DD);
                E0 = f2add(E0, DS);
                E1 = f2add(E1, SS);
                E2 = f2add(E2, DD);
                E3 = f2add(E3, SD);
                sd4(tY, SS, DS, SD, DD);
                E0 = f2add(E0, SD);
                E1 = f2add(E1, DD);
                E2 = f2add(E2, SS);
                E3 = f2add(E3, DS);
                sd4(tZ, SS, DS, SD, DD);
                const float2 U0 = f2mul(wc, f2add(E0, SS)), U1 = f2mul(wc, f2add(E1, DS)), U2 = f2mul(wc, f2add(E2, SD)),
                             U3 = f2mul(wc, f2add(E3, DD));
                const float2 L0 = f2mul(wc, f2sub(E0, SS)), L1 = f2mul(wc, f2sub(E1, DS)), L2 = f2mul(wc, f2sub(E2, SD)),
                             L3 = f2mul(wc, f2sub(E3, DD));
                // faces: in-plane x and y; z from the node's own column
                const float2 pxm = tP[r - 1], pxp = tP[r + 1], vxm = tX[r - 1], vxp = tX[r + 1];
                const float2 pym = tP[r - R::SX], pyp = tP[r + R::SX], vym = tY[r - R::SX], vyp = tY[r + R::SX];
                const float2 fx = f2mul(wf, f2add(f2add(pxp, pxm), f2sub(vxp, vxm)));
                const float2 fy = f2mul(wf, f2add(f2add(pyp, pym), f2sub(vyp, vym)));
                const int m = mrow[s];
                if (s == 0) {
                    const float2 pc = tP[r], vzc = tZ[r];
                    const float2 zd = f2mul(wf, f2add(pc, vzc)), zu = f2mul(wf, f2sub(pc, vzc));
                    const float2 in0 = f2fma(w0, pc, f2add(fx, fy));
                    const float2 in1 = f2mul(wf, f2add(f2sub(pxp, pxm), f2add(vxp, vxm)));
                    const float2 in2 = f2mul(wf, f2add(f2sub(pyp, pym), f2add(vyp, vym)));
                    // completed pair (planes k-1, k): M = L(previous pair) + U(this pair) + in-plane terms, where the
                    // first plane's in-plane terms come from the previous pair and the second's from this one
                    // (components M0, M1x, M1y, M1z, M2xx, M2yy, M2zz, M2xy, M2xz, M2yz)
                    const float2 Uz = f2add(U0, zd), Lz = f2add(L0, zu);
                    float2 Mc[10];
                    Mc[0] = f2add(pL0[4], Uz);
                    Mc[1] = f2add(pL0[1], U1);
                    Mc[2] = f2add(pL0[2], U2);
                    Mc[3] = f2sub(Uz, pL0[4]);
                    Mc[4] = f2add(pL0[0], U0);
                    Mc[5] = f2add(pL0[0], U0);
                    Mc[6] = f2add(pL0[4], Uz);
                    Mc[7] = f2add(pL0[3], U3);
                    Mc[8] = f2sub(U1, pL0[1]);
                    Mc[9] = f2sub(U2, pL0[2]);
                    const float2 In[5] = {in0, in1, in2, fx, fy};
                    const int ic[5] = {0, 1, 2, 4, 5};
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        Mc[ic[t]].x += pI0[t];
                        Mc[ic[t]].y += In[t].x;
                        pI0[t] = In[t].y;
                    }
                    pL0[0] = L0;
                    pL0[1] = L1;
                    pL0[2] = L2;
                    pL0[3] = L3;
                    pL0[4] = Lz;
                    // completed pair: M2 on the halo-1 slot, M0 and M1 of the own column
                    ms[m] = Mc[4];
                    ms[R::NM + m] = Mc[5];
                    ms[2 * R::NM + m] = Mc[7];
                    ms[3 * R::NM + m] = Mc[8];
                    ms[4 * R::NM + m] = Mc[9];
                    ms[5 * R::NM + m] = Mc[6];
                    float2* mo = ms + 6 * R::NM;
                    mo[tid] = Mc[0];
                    mo[R::NT + tid] = Mc[1];
                    mo[2 * R::NT + tid] = Mc[2];
                    mo[3 * R::NT + tid] = Mc[3];
                } else {
                    // the ring node needs the in-plane M2 components xx, yy, xy, xz, yz only
                    float2 Mc[5];
                    Mc[0] = f2add(pL1[0], U0);
                    Mc[1] = f2add(pL1[0], U0);
                    Mc[2] = f2add(pL1[3], U3);
                    Mc[3] = f2sub(U1, pL1[1]);
                    Mc[4] = f2sub(U2, pL1[2]);
                    Mc[0].x += pI1[0];
                    Mc[0].y += fx.x;
                    Mc[1].x += pI1[1];
                    Mc[1].y += fy.x;
                    pI1[0] = fx.y;
                    pI1[1] = fy.y;
                    pL1[0] = L0;
                    pL1[1] = L1;
                    pL1[2] = L2;
                    pL1[3] = L3;
#pragma unroll
                    for (int c = 0; c < 5; ++c) ms[c * R::NM + m] = Mc[c];
                }
            }
        }
        __syncthreads();
        if (j >= 2) {
            float2 u[3] = {f2s(0.f), f2s(0.f), f2s(0.f)}, uc[3] = {f2s(0.f), f2s(0.f), f2s(0.f)};
            {
                const float* up = a.u_prev + gi0;
                const float* uq = a.u_cur + gi0;
                if (ok[0]) {
                    u[0].x = up[0];
                    u[1].x = up[N];
                    u[2].x = up[2 * N];
                }
                if (ok[1]) {
                    u[0].y = up[plane];
                    u[1].y = up[N + plane];
                    u[2].y = up[2 * N + plane];
                }
                if (bzo[0] >= 0) {
                    uc[0].x = uq[0];
                    uc[1].x = uq[N];
                    uc[2].x = uq[2 * N];
                }
                if (bzo[1] >= 0) {
                    uc[0].y = uq[plane];
                    uc[1].y = uq[N + plane];
                    uc[2].y = uq[2 * N + plane];
                }
            }
            // (O) lambda_{n-1} of the pair C_{j-1} = planes (o0, o0 + 1) at the own column
            const float2* ms = mom + ((j - 1) & 1) * R::SLOT;  // C_{j-1}
            const float2* mn = mom + (j & 1) * R::SLOT;        // C_j (its first plane is above the pair)
            const int m = mrow[0];
            const float2 Mxx = ms[m], Myy = ms[R::NM + m], Mxy = ms[2 * R::NM + m], Mxz = ms[3 * R::NM + m],
                         Myz = ms[4 * R::NM + m], Mzz = ms[5 * R::NM + m];
            const float2 M0 = ms[6 * R::NM + tid], M1x = ms[6 * R::NM + R::NT + tid], M1y = ms[6 * R::NM + 2 * R::NT + tid],
                         M1z = ms[6 * R::NM + 3 * R::NT + tid];
            // z-neighbours of the pair's planes: below (zm, .x), above (.y, C_j.x); C_j is empty on the last iteration
            // (its plane lies past the block's planes and only feeds the discarded second lane)
            const bool last = j >= NRP;
            const float nxz = last ? 0.f : mn[3 * R::NM + m].x, nyz = last ? 0.f : mn[4 * R::NM + m].x,
                        nzz = last ? 0.f : mn[5 * R::NM + m].x;
            const float2 zxz = f2(zm[0] - Mxz.y, Mxz.x - nxz), zyz = f2(zm[1] - Myz.y, Myz.x - nyz),
                         zzz = f2(zm[2] - Mzz.y, Mzz.x - nzz);
            zm[0] = Mxz.y;
            zm[1] = Myz.y;
            zm[2] = Mzz.y;
            // sum_a [M2_ab(y - e_a) - M2_ab(y + e_a)] for b = x, y, z
            const float2 dAx = f2add(f2add(f2sub(ms[m - 1], ms[m + 1]), f2sub(ms[2 * R::NM + m - R::MX], ms[2 * R::NM + m + R::MX])), zxz);
            const float2 dAy = f2add(f2add(f2sub(ms[2 * R::NM + m - 1], ms[2 * R::NM + m + 1]),
                                           f2sub(ms[R::NM + m - R::MX], ms[R::NM + m + R::MX])), zyz);
            const float2 dAz = f2add(f2add(f2sub(ms[3 * R::NM + m - 1], ms[3 * R::NM + m + 1]),
                                           f2sub(ms[4 * R::NM + m - R::MX], ms[4 * R::NM + m + R::MX])), zzz);
            // lambda_u = 3 M1 - 3 u M0 + 9 M2 u + A dA
            const float2 m0u = f2mul(cm3, M0);
            float2 v0 = f2fma(c3, M1x, f2fma(m0u, u[0], f2mul(cA, dAx)));
            float2 v1 = f2fma(c3, M1y, f2fma(m0u, u[1], f2mul(cA, dAy)));
            float2 v2 = f2fma(c3, M1z, f2fma(m0u, u[2], f2mul(cA, dAz)));
            v0 = f2fma(c9, f2fma(Mxx, u[0], f2fma(Mxy, u[1], f2mul(Mxz, u[2]))), v0);
            v1 = f2fma(c9, f2fma(Mxy, u[0], f2fma(Myy, u[1], f2mul(Myz, u[2]))), v1);
            v2 = f2fma(c9, f2fma(Mxz, u[0], f2fma(Myz, u[1], f2mul(Mzz, u[2]))), v2);
            const float2 lp = f2mul(c3, M0);
            const float vx[2] = {v0.x, v0.y}, vy[2] = {v1.x, v1.y}, vz[2] = {v2.x, v2.y}, lpp[2] = {lp.x, lp.y};
            const float ux[2] = {u[0].x, u[0].y}, uy[2] = {u[1].x, u[1].y}, uz[2] = {u[2].x, u[2].y};
            const float cx[2] = {uc[0].x, uc[0].y}, cy[2] = {uc[1].x, uc[1].y}, cz[2] = {uc[2].x, uc[2].y};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok[h]) continue;
                const int zo = o0 + h;
                float v[3] = {vx[h], vy[h], vz[h]};
                const bool wzo = !zper && (zo == 0 || zo == nz - 1);
                if (probe_xy && !wzo && zo >= g.probe_lo[2] && zo < g.probe_hi[2]) {
                    const float f = src_factor(a, a.dir[0] * ux[h] + a.dir[1] * uy[h] + a.dir[2] * uz[h]);
#pragma unroll
                    for (int e = 0; e < 3; ++e) v[e] += a.phi_dir[e] * f;
                }
                const int gi = gcol + plane * zo;
                a.lam_out[gi] = lpp[h];
#pragma unroll
                for (int e = 0; e < 3; ++e) a.lam_out[(1 + e) * N + gi] = v[e];
                if (bzo[h] >= 0) {
                    const int bl = bx + g.Fb[0] * (by + g.Fb[1] * bzo[h]);
                    a.boxbuf[3 * Fbn + bl] = cx[h];
                    a.boxbuf[4 * Fbn + bl] = cy[h];
                    a.boxbuf[5 * Fbn + bl] = cz[h];
                }
            }
        }
    }
}

}  // namespace lks
