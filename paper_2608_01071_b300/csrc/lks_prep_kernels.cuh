// Per-call preparation kernels (design and motion parametrisation) and their transposes.
// All in FP64: they touch O(N_d + K + Nt) values once per call.
#pragma once

#include "lks_common.cuh"

namespace lks {

struct DesignGeom {
    int nd[3];       // inner design grid
    int margin;
    int nde[3];      // extended grid
    double R;        // density filter radius (<= 1: identity)
    double beta, eta;
    double kappa_max, q;
};

// Cone weights of Eq. filtering, w = max(0, (R - |d|) / R) for an integer offset d, tabulated by |d|^2 = 0 .. 3 r^2
// (r = floor R <= 32: at most 3073 entries) in shared memory: one square root per entry and block instead of one per
// tap, the FP64 square root being costly on this part.  Every thread of the block must call it.
__device__ __forceinline__ void cone_table(double R, int r, double* sh) {
    const int n = 3 * r * r + 1;
    for (int d2 = threadIdx.x; d2 < n; d2 += blockDim.x) {
        const double w = (R - sqrt((double)d2)) / R;
        sh[d2] = w > 0.0 ? w : 0.0;
    }
    __syncthreads();
}
inline size_t cone_table_bytes(double R) {
    const int r = (int)floor(R);
    return sizeof(double) * (3 * r * r + 1);
}

// Row sums sum_j w_s(i, j) over the design grid (truncated at the edges); static per context.
static __global__ void filter_norm_kernel(DesignGeom dg, double* __restrict__ norm) {
    extern __shared__ double cw[];
    const int r = (int)floor(dg.R);
    cone_table(dg.R, r, cw);
    const long long n = (long long)dg.nd[0] * dg.nd[1] * dg.nd[2];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = i % dg.nd[0], iy = (i / dg.nd[0]) % dg.nd[1], iz = i / ((long long)dg.nd[0] * dg.nd[1]);
    const int rz = dg.nd[2] > 1 ? r : 0;
    double s = 0.0;
    for (int dz = -rz; dz <= rz; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                if (jx < 0 || jx >= dg.nd[0] || jy < 0 || jy >= dg.nd[1] || jz < 0 || jz >= dg.nd[2]) continue;
                s += cw[dx * dx + dy * dy + dz * dz];
            }
    norm[i] = s;
}

// Eq. filtering (transpose = false): out_i = sum_j w_ij in_j / norm_i.
// Transpose (transpose = true):      out_j = sum_i w_ij in_i / norm_i, with `in` already divided by norm
// (filter_scale_kernel), so that no tap divides.  R <= 1 is the identity in both directions.
static __global__ void density_filter_kernel(DesignGeom dg, const double* __restrict__ in, const double* __restrict__ norm,
                                             double* __restrict__ out, int transpose) {
    extern __shared__ double cw[];
    const long long n = (long long)dg.nd[0] * dg.nd[1] * dg.nd[2];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (dg.R <= 1.0) {  // identity (the transposed call then gets its input unscaled)
        if (i < n) out[i] = in[i];
        return;
    }
    const int r = (int)floor(dg.R);
    cone_table(dg.R, r, cw);
    if (i >= n) return;
    const int ix = i % dg.nd[0], iy = (i / dg.nd[0]) % dg.nd[1], iz = i / ((long long)dg.nd[0] * dg.nd[1]);
    const int rz = dg.nd[2] > 1 ? r : 0;
    double s = 0.0;
    for (int dz = -rz; dz <= rz; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                if (jx < 0 || jx >= dg.nd[0] || jy < 0 || jy >= dg.nd[1] || jz < 0 || jz >= dg.nd[2]) continue;
                const double w = cw[dx * dx + dy * dy + dz * dz];
                if (w == 0.0) continue;
                const long long j = jx + (long long)dg.nd[0] * (jy + (long long)dg.nd[1] * jz);
                s += w * in[j];
            }
    out[i] = transpose ? s : s / norm[i];
}

// in / norm, the input of the transposed filter.
static __global__ void filter_scale_kernel(long long n, const double* __restrict__ in, const double* __restrict__ norm,
                                           double* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] / norm[i];
}

// Eq. projection and its derivative; beta = 0 is the identity.
__device__ __forceinline__ double proj(double x, double beta, double eta) {
    if (beta == 0.0) return x;
    return (tanh(beta * eta) + tanh(beta * (x - eta))) / (tanh(beta * eta) + tanh(beta * (1.0 - eta)));
}
__device__ __forceinline__ double proj_d(double x, double beta, double eta) {
    if (beta == 0.0) return 1.0;
    const double c = cosh(beta * (x - eta));
    return beta / (c * c) / (tanh(beta * eta) + tanh(beta * (1.0 - eta)));
}

static __global__ void projection_kernel(long long n, double beta, double eta, const double* __restrict__ in,
                                  double* __restrict__ out, double* __restrict__ dout) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = in[i];
    if (out) out[i] = proj(x, beta, eta);
    if (dout) dout[i] = proj_d(x, beta, eta);
}

// gamma~ -> gamma-bar -> kappa^ref (Eq. kappa_ref) on the extended grid (zero margin), FP64 and state precision.
template <typename T>
__global__ void kappa_ref_kernel(DesignGeom dg, const double* __restrict__ gt, double* __restrict__ gb,
                                 double* __restrict__ kref64, T* __restrict__ kref) {
    const long long ne = (long long)dg.nde[0] * dg.nde[1] * dg.nde[2];
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int ex = e % dg.nde[0], ey = (e / dg.nde[0]) % dg.nde[1], ez = e / ((long long)dg.nde[0] * dg.nde[1]);
    const int m = dg.margin;
    const int mz = dg.nd[2] > 1 ? m : 0;
    const int ix = ex - m, iy = ey - m, iz = ez - mz;
    double k = 0.0;
    if (ix >= 0 && ix < dg.nd[0] && iy >= 0 && iy < dg.nd[1] && iz >= 0 && iz < dg.nd[2]) {
        const long long i = ix + (long long)dg.nd[0] * (iy + (long long)dg.nd[1] * iz);
        const double g = proj(gt[i], dg.beta, dg.eta);
        gb[i] = g;
        k = dg.kappa_max * dg.q * g / ((1.0 - g) + dg.q);
    }
    kref64[e] = k;
    kref[e] = (T)k;
}

// Chain rule: dJ/dkappa^ref (extended grid) -> dJ/dgamma~ on the inner grid (kappa^ref' times projection').
static __global__ void design_chain_kernel(DesignGeom dg, const double* __restrict__ dkref, const double* __restrict__ gt,
                                    const double* __restrict__ gb, double* __restrict__ out) {
    const long long n = (long long)dg.nd[0] * dg.nd[1] * dg.nd[2];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = i % dg.nd[0], iy = (i / dg.nd[0]) % dg.nd[1], iz = i / ((long long)dg.nd[0] * dg.nd[1]);
    const int m = dg.margin;
    const int mz = dg.nd[2] > 1 ? m : 0;
    const long long e = (ix + m) + (long long)dg.nde[0] * ((iy + m) + (long long)dg.nde[1] * (iz + mz));
    const double g = gb[i];
    const double den = (1.0 - g) + dg.q;
    const double dk = dg.kappa_max * dg.q * (1.0 + dg.q) / (den * den);
    out[i] = dkref[e] * dk * proj_d(gt[i], dg.beta, dg.eta);
}

// ------------------------------------------------------------------------------------------------
// Motion (Sec. 2.4): knots at t_k = k Nt / (K - 1); temporal filter of Eq. chi_filtered between knots;
// linear interpolation to every step; u^G_n = s_n - s_{n-1}.
// ------------------------------------------------------------------------------------------------
struct MotionGeom {
    int K, d, Nt;
    double R_t;
};

__device__ __forceinline__ double tri_weight(int k, int m, const MotionGeom& mg) {
    const double tk = (double)k * mg.Nt / (mg.K - 1), tm = (double)m * mg.Nt / (mg.K - 1);
    const double w = (mg.R_t - fabs(tk - tm)) / mg.R_t;
    return w > 0.0 ? w : 0.0;
}

// Row sums sum_m w_km of the temporal filter (static per context).
static __global__ void motion_norm_kernel(MotionGeom mg, double* __restrict__ norm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= mg.K) return;
    double ws = 0.0;
    for (int m = 0; m < mg.K; ++m) ws += tri_weight(k, m, mg);
    norm[k] = ws;
}

// transpose = 0: out_k = sum_m w_km in_m / norm_k.   transpose = 1: out_m = sum_k w_km in_k / norm_k.
static __global__ void motion_filter_kernel(MotionGeom mg, const double* __restrict__ in, const double* __restrict__ norm,
                                     double* __restrict__ out, int transpose) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mg.K * mg.d) return;
    const int k = t / mg.d, a = t % mg.d;
    double s = 0.0;
    for (int m = 0; m < mg.K; ++m) {
        const double w = tri_weight(k, m, mg);
        if (w == 0.0) continue;
        s += transpose ? w * in[m * mg.d + a] / norm[m] : w * in[m * mg.d + a];
    }
    out[t] = transpose ? s : s / norm[k];
}

__device__ __forceinline__ void interp_coef(int n, const MotionGeom& mg, int& k, double& th) {
    const long long num = (long long)n * (mg.K - 1);
    k = (int)(num / mg.Nt);
    if (k > mg.K - 2) k = mg.K - 2;
    th = (double)(num - (long long)k * mg.Nt) / mg.Nt;
}

static __global__ void interp_kernel(MotionGeom mg, const double* __restrict__ f, double* __restrict__ s, double* __restrict__ uG) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (mg.Nt + 1) * mg.d) return;
    const int n = t / mg.d, a = t % mg.d;
    int k;
    double th;
    interp_coef(n, mg, k, th);
    const double sn = (1.0 - th) * f[k * mg.d + a] + th * f[(k + 1) * mg.d + a];
    s[t] = sn;
    // u^G_n = s_n - s_{n-1} (n >= 1), u^G_0 = u^G_1
    const int n1 = n == 0 ? 1 : n;
    int k1, k0;
    double th1, th0;
    interp_coef(n1, mg, k1, th1);
    interp_coef(n1 - 1, mg, k0, th0);
    const double s1 = (1.0 - th1) * f[k1 * mg.d + a] + th1 * f[(k1 + 1) * mg.d + a];
    const double s0 = (1.0 - th0) * f[k0 * mg.d + a] + th0 * f[(k0 + 1) * mg.d + a];
    uG[t] = s1 - s0;
}

// Transpose of interp_kernel: (s-bar, u^G-bar) -> filtered-knot bar.  u^G-bar_0 is ignored (u^G_0 drives no step).
static __global__ void interp_T_kernel(MotionGeom mg, const double* __restrict__ gs, const double* __restrict__ guG,
                                double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mg.K * mg.d) return;
    const int kk = t / mg.d, a = t % mg.d;
    double acc = 0.0;
    // only the steps of the two segments next to knot kk carry its weight
    const int n0 = (int)(((long long)(kk > 0 ? kk - 1 : 0) * mg.Nt) / (mg.K - 1));
    const int n1 = (int)min((long long)mg.Nt, ((long long)(kk + 1) * mg.Nt + mg.K - 2) / (mg.K - 1));
    for (int n = n0; n <= n1; ++n) {
        int k;
        double th;
        interp_coef(n, mg, k, th);
        double c = 0.0;
        if (k == kk) c += 1.0 - th;
        if (k + 1 == kk) c += th;
        if (c == 0.0) continue;
        double g = gs[n * mg.d + a];
        if (n >= 1) g += guG[n * mg.d + a];
        if (n + 1 <= mg.Nt) g -= guG[(n + 1) * mg.d + a];
        acc += c * g;
    }
    out[t] = acc;
}

// Per-step pose: offset o = o0 + s_n, box start and tap weights of the shifted design grid (Eq. rigid_body_position,
// theta = 0; transfer kernel w of Sec. 2.3).  Tap k of a node reads design index j = b - 2 hw + 1 + k, with
// r = t - j = hw - k - f for f = o - floor(o).
// With a rotating body (g.rot), theta_n and omega_n come from `theta` and `omega`, and on x and y the footprint box
// starts at floor(x^G - rb), rb the half extent of the box (the design grid's circumscribed radius plus the kernel's
// half width), with cg = x^G - that start.
static __global__ void pose_kernel(Geom g, int D, double o0x, double o0y, double o0z, int cosine, int Nt,
                            const double* __restrict__ s, const double* __restrict__ uG, const double* __restrict__ theta,
                            const double* __restrict__ omega, double rb, Pose* __restrict__ poses) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n > Nt) return;
    const double o0[3] = {o0x, o0y, o0z};
    Pose P;
    P.pad = 0;
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < 4; ++k) {
            P.w[a][k] = 0.0;
            P.dw[a][k] = 0.0;
        }
        P.xs[a] = 0;
        P.uG[a] = 0.0;
        if (a >= D) continue;
        const double o = o0[a] + s[n * D + a];
        const double oi = floor(o);
        const double f = o - oi;
        int xs = (int)oi - g.hw + 1;
        if (g.periodic[a]) xs = wrap(xs, g.n[a]);
        P.xs[a] = xs;
        P.uG[a] = uG[n * D + a];
        for (int k = 0; k < 2 * g.hw; ++k) {
            const double r = (double)(g.hw - k) - f;
            if (cosine) {
                P.w[a][k] = 0.25 * (1.0 + cos(3.141592653589793 * r / 2.0));
                P.dw[a][k] = (3.141592653589793 / 8.0) * sin(3.141592653589793 * r / 2.0);
            } else {
                P.w[a][k] = k == 0 ? f : 1.0 - f;
                P.dw[a][k] = k == 0 ? 1.0 : -1.0;
            }
        }
    }
    P.th = theta != nullptr ? theta[n] : 0.0;
    P.om = omega != nullptr ? omega[n] : 0.0;
    P.cs[0] = cos(P.th);
    P.cs[1] = sin(P.th);
    P.cg[0] = P.cg[1] = 0.0;
    if (g.rot) {
        for (int a = 0; a < 2; ++a) {
            const double xg = o0[a] + s[n * D + a] + 0.5 * (g.nde[a] - 1);
            const double lo = floor(xg - rb);
            P.cg[a] = xg - lo;
            int xs = (int)lo;
            if (g.periodic[a]) xs = wrap(xs, g.n[a]);
            P.xs[a] = xs;
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < 4; ++k) {
            P.wf[a][k] = (float)P.w[a][k];
            P.dwf[a][k] = (float)P.dw[a][k];
        }
        P.uGf[a] = (float)P.uG[a];
    }
    P.padf = 0.f;
    P.thf = (float)P.th;
    P.omf = (float)P.om;
    for (int a = 0; a < 2; ++a) {
        P.csf[a] = (float)P.cs[a];
        P.cgf[a] = (float)P.cg[a];
    }
    poses[n] = P;
}

// Initial state p' = 0 (p = 1/3), u = 0, wall nodes at their wall velocity.
template <typename T, int D>
__global__ void init_state_kernel(Geom g, T* __restrict__ st) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x[3] = {(int)(i % g.n[0]), (int)((i / g.n[0]) % g.n[1]), (int)(i / ((long long)g.n[0] * g.n[1]))};
    T u[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        if (g.periodic[a]) continue;
        int side = x[a] == 0 ? 0 : (x[a] == g.n[a] - 1 ? 1 : -1);
        if (side >= 0)
            for (int c = 0; c < D; ++c) u[c] = (T)g.wall_u[a][side][c];
    }
    st[i] = 0;
    for (int c = 0; c < D; ++c) st[(1 + c) * g.N + i] = u[c];
}

// Adjoint terminal state: lambda_p = 0, lambda_u = dJ/du_Nt, the objective's source of the last step:
// phi n at the probe nodes, times 1 + 2 phi_var E - 2 phi_var n.u_Nt when the variance term is on (Eq. objective1);
// zero when src = 0.
template <typename T, int D>
__global__ void init_adjoint_kernel(Geom g, const T* __restrict__ u_fin, T* __restrict__ lam, int src) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x[3] = {(int)(i % g.n[0]), (int)((i / g.n[0]) % g.n[1]), (int)(i / ((long long)g.n[0] * g.n[1]))};
    bool wall = false, probe = true;
    for (int a = 0; a < D; ++a) {
        if (!g.periodic[a] && (x[a] == 0 || x[a] == g.n[a] - 1)) wall = true;
        probe = probe && x[a] >= g.probe_lo[a] && x[a] < g.probe_hi[a];
    }
    T f = 1;
    if (probe && !wall && g.phi_var != 0.0) {
        T nu = 0;
        for (int c = 0; c < D; ++c) nu += (T)g.dir[c] * u_fin[c * g.N + i];
        f = (T)g.obj[3] - (T)(2.0 * g.phi_var) * nu;
    }
    lam[i] = 0;
    const bool on = src && probe && !wall;  // src = 0: the objective adds its sources elsewhere (J2)
    for (int c = 0; c < D; ++c) lam[(1 + c) * g.N + i] = on ? (T)(g.dir[c] * g.phi) * f : (T)0;
}

// A state from FP64 host arrays and back: field 0 is stored as p - pshift (pshift = 1/3 for a flow state, whose
// reduced pressure p' = p - 1/3 is kept; 0 for an adjoint state).
template <typename T, int D>
__global__ void import_state_kernel(Geom g, const double* __restrict__ p, const double* __restrict__ u, T* __restrict__ st,
                                    double pshift) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    st[i] = (T)(p[i] - pshift);
    for (int c = 0; c < D; ++c) st[(1 + c) * g.N + i] = (T)u[c * g.N + i];
}

template <typename T, int D>
__global__ void export_state_kernel(Geom g, const T* __restrict__ st, double* __restrict__ p, double* __restrict__ u,
                                    double pshift) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    p[i] = (double)st[i] + pshift;
    for (int c = 0; c < D; ++c) u[c * g.N + i] = (double)st[(1 + c) * g.N + i];
}

// dst += src over all D + 1 fields of a state (the terminal adjoint state of the periodic approximation).
template <typename T, int D>
__global__ void add_state_kernel(Geom g, T* __restrict__ dst, const T* __restrict__ src) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (D + 1) * g.N) return;
    dst[i] += src[i];
}


// One normalised projected-gradient step of the optimiser driver: x_i <- min(hi, max(lo, x_i + step g_i / max|g|))
// NaN into the gradients when the forward sweep they come from raised the stability flag (bit 0 of *flag): the
// asynchronous adjoint cannot return LKS_EUNSTABLE, so its outputs carry the failure instead.
static __global__ void poison_unstable_kernel(const unsigned* __restrict__ flag, double* __restrict__ a, long long na,
                                              double* __restrict__ b, long long nb) {
    if ((flag[0] & 1u) == 0u && flag[1] == 0u) return;  // stable forward and no expired device-side wait
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a != nullptr && i < na) a[i] = __longlong_as_double(0x7ff8000000000000LL);
    if (b != nullptr && i < nb) b[i] = __longlong_as_double(0x7ff8000000000000LL);
}

// (x unchanged where g = 0 everywhere).  A single block: the max-reduction, then the update, so that no scratch
// memory is needed.  Launch with 1024 threads.
static __global__ void __launch_bounds__(1024) gradient_step_kernel(long long n, double step, const double* __restrict__ g,
                                                             double* __restrict__ x, double lo, double hi) {
    __shared__ double red[32];
    double m = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(g[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const double gmax = red[0];
    if (!(gmax > 0.0)) return;
    const double a = step / gmax;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) x[i] = fmin(hi, fmax(lo, x[i] + a * g[i]));
}

}  // namespace lks
