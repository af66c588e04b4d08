// Host runtime of the LKS solver: parameter validation, device memory plan, checkpoint scheduling
// (full storage, sqrt(N) segments, binomial "revolve" schedule) and the C ABI of include/lks.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <initializer_list>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lks.h"
#include "lks_engine.cuh"
#include <map>
#include <tuple>

#include <sys/stat.h>

using namespace lks;

namespace {

// chunks of one step's per-block motion partials summed in parallel before the per-step sums (motion_chunk_kernel)
constexpr int kMotionChunks = 32;

Engine* make_engine(int precision, int D, int hw, const Geom& g) {
    if (D == 2) return precision == LKS_FP64 ? make_engine2d_f64(hw, g) : make_engine2d_f32(hw, g);
    return precision == LKS_FP64 ? make_engine3d_f64(hw, g) : make_engine3d_f32(hw, g);
}

// Binomial coefficient C(c + r, c), saturating.
long long binom_beta(int c, int r) {
    long double v = 1.0L;
    for (int i = 1; i <= c; ++i) {
        v = v * (long double)(r + i) / (long double)i;
        if (v > 1e15L) return (long long)1e15;
    }
    return (long long)(v + 0.5L);
}

// Position of the next checkpoint inside l segments with c free slots (binomial schedule).
int binom_split(int l, int c) {
    int r = 0;
    while (binom_beta(c, r) < l) ++r;
    long long lo = std::max<long long>(1, (long long)l - binom_beta(c - 1, r));
    long long hi = std::min<long long>(l - 1, binom_beta(c, r - 1));
    return (int)std::max(lo, hi);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------------------
struct lks_ctx {
    lks_params prm;
    Geom g;
    DesignGeom dg;
    MotionGeom mg;
    MotionGeom mgw;       // rotating body: the angle knots' filter and interpolation (d = 1, radius R_w)
    bool rot = false;     // the body rotates (K_w > 0)
    bool alks = false;    // the reverse sweep is the ALKS (lks_alks.cuh) instead of the exact discrete adjoint
    void* alam[2] = {nullptr, nullptr};  // ALKS states (1 + D + D(D+1)/2 fields)
    double rb = 0.0;      // half extent of the rotating body's footprint box on x and y
    int D = 2, hw = 1, cosine = 0;
    double o0[3] = {0, 0, 0};
    size_t tsize = 8;
    std::unique_ptr<Engine> eng;
    int max_ablocks = 0;  // most adjoint blocks over all tile choices (motion-slot stride)
    int max_njb = 0;      // most probe blocks over all tile choices (objective-slot stride)
    bool oar = false;     // the objective is J2 of Eq. objective2 (translating body)
    OarGeom ogeo{};
    int nbox = 0;         // blocks of the footprint-box kernels (objective J2 scratch stride)
    double *d_oslot = nullptr, *d_oms = nullptr, *d_oar_guG = nullptr, *d_oar_dK = nullptr;
    // J2 with a rotating body: compensated d j2 / d kappa^ref (state precision, nde each), K / M1 / I, per-step
    // d/dtheta and d/domega, and the scratch of the constants' last-block sum
    void *d_okh = nullptr, *d_okl = nullptr;
    double *d_ocst = nullptr, *d_ocscr = nullptr, *d_oar_gth = nullptr, *d_oar_gom = nullptr;
    double *d_oscr = nullptr, *d_omsscr = nullptr;  // per-block partials of one step (J2 forward / sensitivities)
    unsigned* d_otick = nullptr;  // last-block tickets: [0] forward, [1 + s] sensitivity step s, [Lmax + 1] constants
    long long nd = 0, nde = 0;
    std::string err;
    lks_stats stats;

    // device memory
    std::vector<void*> allocs;
    double* d_fscr = nullptr;  // nd: the transposed filter's input divided by the row sums
    double *d_gamma = nullptr, *d_gt = nullptr, *d_gb = nullptr, *d_kref64 = nullptr, *d_fnorm = nullptr,
           *d_tmp = nullptr;
    void* d_kref = nullptr;
    double *d_knots = nullptr, *d_filt = nullptr, *d_s = nullptr, *d_uG = nullptr, *d_ktmp = nullptr;
    double *d_out_g = nullptr, *d_out_k = nullptr;  // host-pointer adjoint staging
    double* d_tnorm = nullptr;                        // temporal-filter row sums
    // rotating body: angle knots, filtered knots and filter row sums, theta_n, omega_n, their sensitivities, the
    // angle-knot gradient, and the step's kappa, u^S on the footprint box
    double *d_aknots = nullptr, *d_afilt = nullptr, *d_anorm = nullptr, *d_theta = nullptr, *d_omega = nullptr,
           *d_gth = nullptr, *d_gom = nullptr, *d_atmp = nullptr, *d_out_a = nullptr;
    void* d_rotmap = nullptr;
    Pose* d_pose = nullptr;
    double *d_gs = nullptr, *d_guG = nullptr, *d_dkref = nullptr, *d_jslot = nullptr, *d_jstep = nullptr,
           *d_J = nullptr;
    unsigned* d_flag = nullptr;
    unsigned* h_flag = nullptr;  // pinned
    cudaEvent_t ev_flag = nullptr;
    void* d_kbar = nullptr;
    double* d_mslot = nullptr;
    double* d_mpart = nullptr;  // Lmax steps x kMotionChunks chunk sums of d_mslot
    void* d_boxbuf = nullptr;   // two buffers of Lmax steps x 2D planes x Fbn (lam_u, u_n on the footprint box)
    long long box_step = 0;     // elements per step in d_boxbuf
    void* d_fac = nullptr;      // two buffers of Lmax steps x Fbn: 1 / (1 + kappa) on the footprint box
    bool throughput = false;    // instance of a batch: tune for throughput (see create_ctx)
    void* d_init = nullptr;     // caller's initial state (lks_set_initial_state), in the state layout
    bool custom_init = false;
    void* d_lterm = nullptr;    // caller's terminal adjoint state (lks_set_adjoint_terminal), in the state layout
    bool custom_lterm = false;
    bool have_lambda0 = false;  // lam[0] holds lambda_0 of the last adjoint
    // step-kernel variants of the forward sweep, the recomputation and the adjoint steps (see choose_variants)
    int rows_fwd_sweep = 0, rows_rec = 0, rows_adj = 0;
    // tuner results: fastest forward / adjoint variant alone, and the fastest one-step pair run side by side
    int tune_f_lat = 0, tune_f_one = 0, tune_a_lat = 0, tune_a_one = 0;
    int nsb = 0;                // sensitivity blocks per step
    size_t state_bytes = 0;
    std::vector<void*> slot;  // checkpoint slots
    std::vector<void*> hist[2];  // recompute history, two buffers (index 0 unused)
    std::vector<const void*> seg_st[2];  // where the states of the segment in each buffer live
    cudaStream_t side = nullptr, cap2 = nullptr;   // recompute chain (eager / capture)
    cudaStream_t side2 = nullptr, cap3 = nullptr;  // sensitivity chain (eager / capture)
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr}, ev_sens[2] = {nullptr, nullptr};
    cudaEvent_t ev_sync[3] = {nullptr, nullptr, nullptr};
    void* pp[3] = {nullptr, nullptr, nullptr};
    void* tmp_state = nullptr;
    void* fin = nullptr;
    void* lam[2] = {nullptr, nullptr};

    // schedule
    int S = 1;             // boundary spacing (segment length)
    int M = 1;             // number of segments
    int Lmax = 1;          // longest segment (sensitivity buffer depth)
    int fac_written[2] = {0, 0};  // per history buffer: leading steps whose 1 / (1 + kappa) the recompute wrote
    int free_slots = 0;    // REVOLVE: slots besides boundary 0
    // the reverse sweep pipelines recomputation, adjoint and sensitivities on three streams with two history buffers:
    // SQRT, and REVOLVE when the slots hold every segment boundary (the binomial schedule is then the sqrt one)
    bool pipelined = false;
    std::vector<int> chain;  // REVOLVE: boundaries stored by the forward sweep (after 0)
    std::vector<int> slot_of;  // boundary -> slot index or -1
    std::vector<int> slot_used;

    bool have_forward = false;
    bool have_final = false;  // the final-state buffer holds the last forward's state (the reverse sweeps never write it)
    long long launches = 0;
    long long launches_fwd = 0, launches_adj = 0;

    // CUDA graphs of the forward sweep and of the reverse sweep (captured once, replayed every call)
    bool use_graphs = true;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gx_fwd = nullptr, gx_adj = nullptr;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans_fwd, spans_adj;

    // optional CUDA-event timing of the step kernels
    bool timing = false;
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;  // (kind, (start, end))
    cudaEvent_t ev_all0 = nullptr, ev_end = nullptr;

    int step_of(int m) const { return std::min(m * S, prm.Nt); }
    void* state_ptr_stored(int m) const {  // state of boundary m if stored
        if (m == M) return fin;
        int si = slot_of[m];
        return si >= 0 ? slot[si] : nullptr;
    }
    char* tptr(void* p, long long off) const { return (char*)p + off * (long long)tsize; }
};

namespace {

void set_err(lks_ctx* c, const LksError& e) {
    if (c) c->err = e.msg;
}

void* dalloc(lks_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw LksError{LKS_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
    }
    c->allocs.push_back(p);
    c->stats.device_bytes += (int64_t)bytes;
    return p;
}

void validate(const lks_params* p) {
    auto bad = [](const std::string& m) { throw LksError{LKS_EINVAL, m}; };
    if (!p) bad("params is NULL");
    if (p->size != sizeof(lks_params)) bad("params.size does not match this library's lks_params");
    if (p->lattice != LKS_D2Q9 && p->lattice != LKS_D3Q15) bad("lattice must be LKS_D2Q9 or LKS_D3Q15");
    const int D = p->lattice == LKS_D2Q9 ? 2 : 3;
    for (int a = 0; a < 3; ++a) {
        if (a < D && (p->n[a] < 4 || p->n[a] > (1 << 20))) bad("grid extent out of range [4, 2^20]");
        if (a >= D && p->n[a] != 1) bad("n[2] must be 1 for D2Q9");
        if (a < D && (p->nd[a] < 1)) bad("design extent must be >= 1");
        if (a >= D && p->nd[a] != 1) bad("nd[2] must be 1 for D2Q9");
    }
    long long N = (long long)p->n[0] * p->n[1] * p->n[2];
    if (N > (1LL << 31)) bad("grid too large");
    if (!(p->nu > 0.0) || !(p->nu < 1.0)) bad("nu must be in (0, 1)");
    if (!(p->kappa_max >= 0.0) || !(p->q > 0.0)) bad("kappa_max >= 0 and q > 0 required");
    if (p->margin < 0 || p->margin > 64) bad("margin out of range");
    if (p->map_kernel != LKS_MAP_LINEAR && p->map_kernel != LKS_MAP_COSINE) bad("unknown map_kernel");
    const int hw = p->map_kernel == LKS_MAP_LINEAR ? 1 : 2;
    for (int a = 0; a < D; ++a) {
        const int nde = p->nd[a] + 2 * p->margin;
        if (p->periodic[a] && nde + 2 * hw > p->n[a])
            bad("design grid plus kernel support must fit in one period of a periodic axis");
        if (p->probe_lo[a] < 0 || p->probe_hi[a] > p->n[a] || p->probe_lo[a] >= p->probe_hi[a])
            bad("probe box must satisfy 0 <= lo < hi <= n");
    }
    if (p->Nt < 1 || p->Nt > 10000000) bad("Nt out of range");
    if (p->K < 2 || p->K > 1000000) bad("K must be >= 2");
    if (!(p->R_t > 0.0)) bad("R_t must be > 0");
    if (!(p->filter_R >= 0.0) || p->filter_R > 32.0) bad("filter_R out of range [0, 32]");
    if (!(p->beta >= 0.0) || !(p->eta > 0.0 && p->eta < 1.0)) bad("beta >= 0 and 0 < eta < 1 required");
    if (p->precision != LKS_FP64 && p->precision != LKS_FP32) bad("unknown precision");
    if (p->ckpt < LKS_CKPT_FULL || p->ckpt > LKS_CKPT_REVOLVE) bad("unknown ckpt");
    if (p->mode < LKS_MODE_JOINT || p->mode > LKS_MODE_MOTION) bad("unknown mode");
    if (p->ckpt_slots < 0 || p->seg_len < 0 || p->ckpt_bytes < 0) bad("negative checkpoint setting");
    if (!std::isfinite(p->phi_var)) bad("phi_var must be finite");
    if (p->objective != LKS_OBJ_FLOW && p->objective != LKS_OBJ_OAR) bad("unknown objective");
    if (p->adjoint != LKS_ADJ_DISCRETE && p->adjoint != LKS_ADJ_ALKS) bad("unknown adjoint");
    if (p->adjoint == LKS_ADJ_ALKS && (p->objective != LKS_OBJ_FLOW || p->phi_var != 0.0 || p->K_w != 0))
        bad("the ALKS reverse sweep is built for objective LKS_OBJ_FLOW with phi_var = 0 and a translating body");
    if (p->K_w != 0) {
        if (p->K_w < 2 || p->K_w > 1000000) bad("K_w must be 0 (no rotation) or >= 2 angle knots");
        if (!(p->R_w > 0.0)) bad("R_w must be > 0 with a rotating body");
        if (p->objective == LKS_OBJ_OAR && (!(p->l_m > 0.0) || !std::isfinite(p->l_m) || !std::isfinite(p->w_T)))
            bad("J2 with a rotating body needs l_m > 0 and a finite w_T");
        if (p->tile_rows > 1 || p->tile_rows_rec > 1)
            bad("with a rotating body the forward sweep runs step-kernel variant 1 (tile_rows 0 or 1)");
    }
    if (p->objective == LKS_OBJ_OAR) {
        if (!(p->drag_span > 0.0) || !std::isfinite(p->drag_span) || !std::isfinite(p->w_D))
            bad("objective J2 needs drag_span > 0 and a finite w_D");
        if (p->phi_var != 0.0) bad("phi_var belongs to objective J1");
    }
    // a step-kernel variant code: the forward accepts 3 (two steps per launch), the adjoint does not
    auto variant_ok = [&](int r, bool fwd) {
        if (D == 3)
            return r == 1 || r == 8 || r == 16 || r == 32 || r == 64 || (fwd && r == 96) ||
                   ((r == 128 || r == 160 || (!fwd && r == 192)) && p->precision == LKS_FP32);
        return r == 1 || r == 2 || r == 3 || r == 4 || r == 8 || (r == 16 && p->precision == LKS_FP32) ||
               ((r == 32 || r == 64) && p->n[0] % 2 == 0);
    };
    if (p->tile_rows != 0 && !variant_ok(p->tile_rows, true))
        bad(D == 2 ? "D2Q9 tile_rows must be 0 (autotune), 1 or 2 (row tiles), 3 (two-step row tiles), 4, 8, "
                     "16 (FP32) or 32, 64 (even nx)"
                   : "D3Q15 tile_rows must be 0 (autotune), 1 (shared-memory tiles), 8 or 16 (z planes per block), "
                     "32, 64 (separable, 16 or 32 planes per block), 96 (separable forward, 16 x 16 columns), "
                     "128, 160 (plane-pair separable kernels, FP32, 16 or 32 planes per block)");
    if (p->tile_rows_adj != 0 && (p->tile_rows == 0 || !variant_ok(p->tile_rows_adj, false)))
        bad("tile_rows_adj must be 0, or a valid adjoint variant with tile_rows != 0 (D3Q15 FP32 also 192: plane-pair "
            "adjoint with 64 planes per block)");
    if (p->tile_rows_rec != 0 && (p->tile_rows == 0 || !variant_ok(p->tile_rows_rec, true)))
        bad("tile_rows_rec must be 0, or a valid forward variant with tile_rows != 0");
}

void setup_geometry(lks_ctx* c) {
    const lks_params& p = c->prm;
    c->D = p.lattice == LKS_D2Q9 ? 2 : 3;
    c->hw = p.map_kernel == LKS_MAP_LINEAR ? 1 : 2;
    c->cosine = p.map_kernel == LKS_MAP_COSINE;
    c->tsize = p.precision == LKS_FP64 ? 8 : 4;
    Geom& g = c->g;
    std::memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a) {
        g.n[a] = p.n[a];
        g.periodic[a] = a < c->D ? (p.periodic[a] ? 1 : 0) : 1;
        g.nde[a] = a < c->D ? p.nd[a] + 2 * p.margin : 1;
        g.Fb[a] = a < c->D ? g.nde[a] + 2 * c->hw - 1 : 1;
        g.probe_lo[a] = a < c->D ? p.probe_lo[a] : 0;
        g.probe_hi[a] = a < c->D ? p.probe_hi[a] : 1;
        g.dir[a] = a < c->D ? p.direction[a] : 0.0;
        for (int s = 0; s < 2; ++s)
            for (int b = 0; b < 3; ++b) g.wall_u[a][s][b] = p.wall_velocity[a][s][b];
    }
    g.N = (long long)p.n[0] * p.n[1] * p.n[2];
    g.hw = c->hw;
    g.Fbn = (long long)g.Fb[0] * g.Fb[1] * g.Fb[2];
    g.A = 0.75 - 4.5 * p.nu;
    g.u_crit2 = p.u_crit > 0.0 ? p.u_crit * p.u_crit : 0.0;
    // limit of the bounded device-side waits, and the diagnostic that makes them expire
    if (const char* e = std::getenv("LKS_WAIT_NS"); e && *e) g.wait_ns = std::strtoull(e, nullptr, 10);
    if (const char* e = std::getenv("LKS_WAIT_PROBE"); e && *e) g.wait_probe = std::atoi(e) != 0 ? 1 : 0;
    // |O| counts probe nodes off the walls
    long long cnt = 1;
    for (int a = 0; a < c->D; ++a) {
        int lo = p.probe_lo[a], hi = p.probe_hi[a];
        if (!g.periodic[a]) {
            lo = std::max(lo, 1);
            hi = std::min(hi, p.n[a] - 1);
        }
        cnt *= std::max(0, hi - lo);
    }
    if (cnt <= 0) throw LksError{LKS_EINVAL, "probe box holds no fluid node"};
    g.phi = 1.0 / ((double)p.Nt * (double)cnt);
    g.phi_var = p.phi_var;
    const double nD = (double)p.nd[0] * p.nd[1] * p.nd[2];
    c->oar = p.objective == LKS_OBJ_OAR;
    c->ogeo.cL = 1.0 / ((double)p.Nt * nD);
    c->ogeo.cD = c->oar ? p.w_D / (p.drag_span * nD) : 0.0;
    c->ogeo.cT = c->oar && p.K_w > 0 ? p.w_T / (2.0 * M_PI * p.l_m * nD) : 0.0;
    for (int a = 0; a < c->D; ++a) {
        const double center = std::isnan(p.base_center[a]) ? (p.n[a] - 1) / 2.0 : p.base_center[a];
        c->o0[a] = center - (g.nde[a] - 1) / 2.0;
    }
    DesignGeom& dg = c->dg;
    for (int a = 0; a < 3; ++a) {
        dg.nd[a] = p.nd[a];
        dg.nde[a] = g.nde[a];
    }
    dg.margin = p.margin;
    dg.R = p.filter_R;
    dg.beta = p.beta;
    dg.eta = p.eta;
    dg.kappa_max = p.kappa_max;
    dg.q = p.q;
    c->mg.K = p.K;
    c->mg.d = c->D;
    c->mg.Nt = p.Nt;
    c->mg.R_t = p.R_t;
    c->rot = p.K_w > 0;
    c->alks = p.adjoint == LKS_ADJ_ALKS;
    g.rot = c->rot ? 1 : 0;
    if (c->rot) {
        // footprint box on x and y: the design grid's circumscribed circle around x^G plus the kernel's half width
        const double hx = 0.5 * (g.nde[0] - 1), hy = 0.5 * (g.nde[1] - 1);
        c->rb = std::sqrt(hx * hx + hy * hy) + c->hw;
        for (int a = 0; a < 2; ++a) {
            g.Fb[a] = (int)std::ceil(2.0 * c->rb) + 2;
            if (g.periodic[a] && g.Fb[a] > p.n[a])
                throw LksError{LKS_EINVAL, "the rotating body's footprint must fit in one period of a periodic axis"};
        }
        g.Fbn = (long long)g.Fb[0] * g.Fb[1] * g.Fb[2];
        c->mgw.K = p.K_w;
        c->mgw.d = 1;
        c->mgw.Nt = p.Nt;
        c->mgw.R_t = p.R_w;
    }
    c->nd = (long long)p.nd[0] * p.nd[1] * p.nd[2];
    c->nde = (long long)g.nde[0] * g.nde[1] * g.nde[2];
    // the mapping and sensitivity kernels index the design grid and the footprint-box records in 32 bits
    if (c->nde >= (1LL << 31) || 6 * g.Fbn >= (1LL << 31))
        throw LksError{LKS_EINVAL, "design grid or footprint box too large (2^31 design nodes, 2^31 / 6 box nodes)"};
}

// Checkpoint layout: boundaries every S steps; FULL keeps every state, SQRT every ceil(sqrt Nt)-th,
// REVOLVE keeps boundary 0 plus a binomial schedule over M segments of length S with free_slots slots.
void plan_checkpoints(lks_ctx* c, size_t state_bytes) {
    const lks_params& p = c->prm;
    const int Nt = p.Nt;
    if (p.ckpt == LKS_CKPT_FULL) {
        c->S = 1;
    } else if (p.seg_len > 0) {
        c->S = std::min(p.seg_len, Nt);
    } else {
        c->S = std::max(1, (int)std::ceil(std::sqrt((double)Nt)));
    }
    c->M = (Nt + c->S - 1) / c->S;
    c->Lmax = p.ckpt == LKS_CKPT_FULL ? std::min(Nt, 256) : c->S;
    int nslots;
    if (p.ckpt == LKS_CKPT_REVOLVE) {
        int freec = p.ckpt_slots;
        if (freec == 0) {
            // budget: slots + history (S + 1) + 2 ping-pong + tmp + final + 2 adjoint states
            long long fixed = (long long)(c->S + 1 + 2 + 1 + 1 + 2) * (long long)state_bytes;
            long long avail = p.ckpt_bytes > 0 ? p.ckpt_bytes - fixed : 0;
            freec = (int)std::max<long long>(1, avail / (long long)state_bytes - 1);
        }
        // every boundary fits, and (under a byte budget) so does a second history buffer: pipeline the sweep
        c->pipelined = c->M > 1 && freec >= c->M - 1 && (p.ckpt_slots > 0 || freec >= c->M - 1 + c->S);
        freec = std::max(1, std::min(freec, c->M - 1 > 0 ? c->M - 1 : 1));
        c->free_slots = freec;
        nslots = 1 + freec;
        // right spine of the recursion: boundaries the forward sweep stores
        c->chain.clear();
        int a = 0, b = c->M, f = freec;
        while (b - a > 1 && f > 0) {
            int m = a + binom_split(b - a, f);
            c->chain.push_back(m);
            a = m;
            --f;
        }
    } else {
        // FULL: every state; SQRT: boundaries 0, S, 2S, ... below Nt
        nslots = c->M;
        c->pipelined = p.ckpt == LKS_CKPT_SQRT;
    }
    c->slot_of.assign(c->M + 1, -1);
    c->slot_used.assign(nslots, 0);
    (void)nslots;
}

int njb_of(const lks_ctx* c);

// Size the slot strides for every tile choice the autotuner may make, then start from the default tiles.
void choose_rows_initial(lks_ctx* c) {
    c->max_ablocks = 0;
    c->max_njb = 0;
    const std::vector<int> cf = c->eng->fwd_codes(), ca = c->eng->adj_codes();
    for (int rf : cf)
        for (int ra : ca) {
            if (!c->eng->set_rows(rf, ra, c->g)) continue;
            const dim3 ag = c->eng->agrid;
            c->max_ablocks = std::max(c->max_ablocks, (int)(ag.x * ag.y * ag.z));
            c->max_njb = std::max(c->max_njb, njb_of(c));
        }
    // a rotating body's forward runs variant 1 (the step kernel that reads the rotated footprint map)
    const int r = c->prm.tile_rows > 0 ? c->prm.tile_rows : (c->D == 2 || c->rot ? 1 : 8);
    int ra = c->prm.tile_rows_adj > 0 ? c->prm.tile_rows_adj : r;
    if (c->prm.tile_rows_adj <= 0 && std::find(ca.begin(), ca.end(), ra) == ca.end()) ra = c->D == 2 ? 1 : 8;
    if (!c->eng->set_rows(r, ra, c->g)) throw LksError{LKS_EINVAL, "step-kernel variant not available for this grid"};
}

// Tile autotuner (D2Q9): time the forward and adjoint step kernels for every rows-per-warp choice on the
// context's own buffers and keep the fastest of each.  Results are cached per (device, precision, kernel
// width, grid) for the life of the process.
// The tuner's choices decide which step kernels run, and the kernels of one lattice differ in the order of their FP
// additions: two processes that tuned separately could return gradients that differ in the last bits.  The choices
// are therefore also kept in a file, one line per (device model, precision, transfer kernel, lattice, grid), read
// before tuning and appended after it, so that every process on a machine runs the same kernels.  The file is
// $LKS_TUNE_FILE (an empty value: no file), else $XDG_CACHE_HOME/lks/tune.txt, else $HOME/.cache/lks/tune.txt.
std::string tune_file_path() {
    const char* f = std::getenv("LKS_TUNE_FILE");
    if (f) return std::string(f);
    std::string dir;
    if (const char* x = std::getenv("XDG_CACHE_HOME"); x && *x)
        dir = x;
    else if (const char* h = std::getenv("HOME"); h && *h)
        dir = std::string(h) + "/.cache";
    else
        return std::string();
    mkdir(dir.c_str(), 0755);
    dir += "/lks";
    mkdir(dir.c_str(), 0755);
    return dir + "/tune.txt";
}

std::string tune_key(const lks_ctx* c, int dev) {
    cudaDeviceProp prop;
    LKS_CUDA(cudaGetDeviceProperties(&prop, dev));
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "v%d|%s|sm%d%d|t%d|hw%d|d%d|rot%d|%dx%dx%d", LKS_ABI_VERSION * 100 + 4, name.c_str(),
                  prop.major, prop.minor, (int)c->tsize, c->hw, c->D, c->rot ? 1 : 0, c->g.n[0], c->g.n[1], c->g.n[2]);
    return buf;
}

bool tune_file_read(const std::string& path, const std::string& key, std::array<int, 4>& out) {
    if (path.empty()) return false;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {  // the last matching line wins
        char k[320];
        int v[4];
        if (std::sscanf(line, "%319s %d %d %d %d", k, &v[0], &v[1], &v[2], &v[3]) == 5 && key == k) {
            out = {v[0], v[1], v[2], v[3]};
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_file_append(const std::string& path, const std::string& key, const std::array<int, 4>& v) {
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return;  // a cache: the choices still hold for this process
    std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3]);
    std::fclose(f);
}

void autotune_rows(lks_ctx* c) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int>, std::array<int, 4>> cache;
    int dev = 0;
    LKS_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, (int)c->tsize, c->hw * 16 + c->D + (c->rot ? 64 : 0), c->g.n[0],
                                     c->g.n[1] * 65536 + c->g.n[2]);
    const std::string fkey = tune_key(c, dev), fpath = tune_file_path();
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        std::array<int, 4> v;
        if (it == cache.end() && tune_file_read(fpath, fkey, v)) {
            // choices of an earlier process, kept only if this version of the library still offers them on this grid
            const int rf0 = c->eng->rows_f, ra0 = c->eng->rows_a;
            if (c->eng->set_rows(v[0], v[2], c->g) && c->eng->set_rows(v[1], v[3], c->g)) it = cache.emplace(key, v).first;
            c->eng->set_rows(rf0, ra0, c->g);
        }
        if (it != cache.end()) {
            c->tune_f_lat = it->second[0];
            c->tune_f_one = it->second[1];
            c->tune_a_lat = it->second[2];
            c->tune_a_one = it->second[3];
            return;
        }
    }
    cudaStream_t s = c->side;
    LKS_CUDA(cudaMemsetAsync(c->d_pose, 0, 2 * sizeof(Pose), s));  // poses 0 and 1 (Nt >= 1)
    LKS_CUDA(cudaMemsetAsync(c->lam[0], 0, c->state_bytes, s));
    LKS_CUDA(cudaMemsetAsync(c->lam[1], 0, c->state_bytes, s));
    c->eng->init_state(c->g, c->slot[0], s);
    c->eng->init_state(c->g, c->pp[2], s);
    cudaEvent_t e0, e1;
    LKS_CUDA(cudaEventCreate(&e0));
    LKS_CUDA(cudaEventCreate(&e1));
    // every forward variant with the initial adjoint one, then every adjoint variant with the initial forward one
    const std::vector<int> cf = c->eng->fwd_codes(), ca = c->eng->adj_codes();
    const int rf0 = c->eng->rows_f, ra0 = c->eng->rows_a;
    // fastest overall, for each kernel; the one-step variants' times are kept for the pair timing below
    float best_f = 1e30f, best_a = 1e30f;
    int rf = rf0, ra = ra0;
    std::vector<std::pair<float, int>> one_f, one_a;
    const int jlo[3] = {0, 0, 0}, jn[3] = {1, 1, 1};
    // ms per step of `reps` back-to-back launches of one variant after 3 untimed ones
    auto time_variant = [&](int r, int pass, int reps) {
        for (int k = 0; k < 3 + reps; ++k) {
            if (k == 3) LKS_CUDA(cudaEventRecord(e0, s));
            if (pass == 0 && c->eng->fused2())
                c->eng->fwd2(c->g, c->slot[0], c->pp[0], c->pp[1], c->d_kref, c->d_pose, nullptr, nullptr, c->d_flag,
                             jlo, jn, s);
            else if (pass == 0)
                c->eng->fwd(c->g, c->slot[0], c->pp[k & 1], c->d_kref, c->d_pose, nullptr, c->d_flag, jlo, jn, s);
            else if (c->eng->fused_adj2())
                c->eng->adj2(c->g, c->lam[k & 1], c->lam[(k + 1) & 1], c->slot[0], c->slot[0], c->slot[0], c->d_kref,
                             c->d_pose + 1, c->d_boxbuf, c->d_fac, 1, c->d_boxbuf, c->d_fac, 1, s);
            else  // u_{n-1} and u_n from different buffers, as in the reverse sweep (the footprint records read u_n)
                c->eng->adj(c->g, c->lam[k & 1], c->lam[(k + 1) & 1], c->slot[0], c->pp[2], c->d_kref, c->d_pose,
                            c->d_boxbuf, c->d_fac, 1, s);
        }
        LKS_CUDA(cudaEventRecord(e1, s));
        LKS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LKS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        // the fused variant takes two steps per launch
        return ms / (float)reps / ((pass == 0 ? c->eng->fused2() : c->eng->fused_adj2()) ? 2.f : 1.f);
    };
    // Each variant is first sized to about 1.5 ms of launches; then three rounds time every variant once per round
    // and keep each one's fastest.  Rounds rather than back-to-back trials spread a drift of the clocks over all
    // candidates instead of favouring the ones timed last.
    for (int pass = 0; pass < 2; ++pass) {
        struct Cand { int r; int reps; float ms; bool one_step; };
        std::vector<Cand> cands;
        for (int r : (pass == 0 ? cf : ca)) {
            if (pass == 0 && c->rot && r != 1) continue;  // a rotating body's forward runs variant 1
            // not available for this grid / precision
            if (!(pass == 0 ? c->eng->set_rows(r, ra0, c->g) : c->eng->set_rows(rf0, r, c->g))) continue;
            const float est = time_variant(r, pass, 10);
            cands.push_back({r, std::max(10, std::min(2000, (int)(1.5f / std::max(est, 1e-4f)))), est,
                             pass == 0 ? !c->eng->fused2() : !c->eng->fused_adj2()});
        }
        for (int trial = 0; trial < 3; ++trial)
            for (Cand& k : cands) {
                if (!(pass == 0 ? c->eng->set_rows(k.r, ra0, c->g) : c->eng->set_rows(rf0, k.r, c->g)))
                    throw LksError{LKS_ECUDA, "internal: tuner variant became unavailable"};
                k.ms = std::min(k.ms, time_variant(k.r, pass, k.reps));
            }
        for (const Cand& k : cands) {
            if (std::getenv("LKS_TUNE_VERBOSE"))
                std::fprintf(stderr, "lks autotune %dx%dx%d %s rows=%d: %.3f us/step (%d launches)\n", c->g.n[0],
                             c->g.n[1], c->g.n[2], pass == 0 ? "forward" : "adjoint", k.r, 1e3f * k.ms, k.reps);
            if (pass == 0 && k.ms < best_f) {
                best_f = k.ms;
                rf = k.r;
            }
            if (pass == 1 && k.ms < best_a) {
                best_a = k.ms;
                ra = k.r;
            }
            if (k.one_step) (pass == 0 ? one_f : one_a).push_back({k.ms, k.r});
        }
    }
    // Chains that share the GPU (the recomputation beside the adjoint chain): time the three fastest one-step
    // forward variants against the three fastest one-step adjoint variants, launched together on two streams,
    // and keep the pair with the shortest time per step of both.  Isolated timings do not rank these well: on
    // 512x256 the 16-row forward and adjoint tiles are faster alone and slower together.
    std::sort(one_f.begin(), one_f.end());
    std::sort(one_a.begin(), one_a.end());
    if (one_f.size() > 3) one_f.resize(3);
    if (one_a.size() > 3) one_a.resize(3);
    cudaStream_t s2 = c->side2;
    cudaEvent_t e2;
    LKS_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    auto time_pair = [&](int reps) {
        for (int k = 0; k < 3 + reps; ++k) {
            if (k == 3) {
                LKS_CUDA(cudaStreamSynchronize(s2));
                LKS_CUDA(cudaEventRecord(e0, s));
                LKS_CUDA(cudaStreamWaitEvent(s2, e0, 0));
            }
            c->eng->fwd(c->g, c->slot[0], c->pp[k & 1], c->d_kref, c->d_pose, nullptr, c->d_flag, jlo, jn, s2);
            c->eng->adj(c->g, c->lam[k & 1], c->lam[(k + 1) & 1], c->slot[0], c->pp[2], c->d_kref, c->d_pose,
                        c->d_boxbuf, c->d_fac, 1, s);
        }
        LKS_CUDA(cudaEventRecord(e2, s2));
        LKS_CUDA(cudaStreamWaitEvent(s, e2, 0));
        LKS_CUDA(cudaEventRecord(e1, s));
        LKS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LKS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms / (float)reps;
    };
    float best_pair = 1e30f;
    int rf1 = one_f.empty() ? rf0 : one_f[0].second, ra1 = one_a.empty() ? ra0 : one_a[0].second;
    struct Pair { int f, a, reps; float ms; };
    std::vector<Pair> pairs;
    for (const auto& f : one_f)
        for (const auto& ad : one_a)
            if (c->eng->set_rows(f.second, ad.second, c->g))
                pairs.push_back({f.second, ad.second,
                                 std::max(10, std::min(2000, (int)(1.5f / std::max(f.first + ad.first, 1e-4f)))), 1e30f});
    // three rounds over all pairs, as for the single variants
    for (int trial = 0; trial < 3; ++trial)
        for (Pair& q : pairs) {
            if (!c->eng->set_rows(q.f, q.a, c->g)) throw LksError{LKS_ECUDA, "internal: tuner pair became unavailable"};
            q.ms = std::min(q.ms, time_pair(q.reps));
        }
    for (const Pair& q : pairs) {
        if (std::getenv("LKS_TUNE_VERBOSE"))
            std::fprintf(stderr, "lks autotune %dx%dx%d forward rows=%d beside adjoint rows=%d: %.3f us/step\n",
                         c->g.n[0], c->g.n[1], c->g.n[2], q.f, q.a, 1e3f * q.ms);
        if (q.ms < best_pair) {
            best_pair = q.ms;
            rf1 = q.f;
            ra1 = q.a;
        }
    }
    cudaEventDestroy(e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_f_lat = rf;
    c->tune_f_one = rf1;
    c->tune_a_lat = ra;
    c->tune_a_one = ra1;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = {rf, rf1, ra, ra1};
    tune_file_append(fpath, fkey, cache[key]);
}

// Variants of the three kinds of step launches.  The forward sweep is one chain, so it takes the fastest
// variant.  In the pipelined sqrt(N) reverse sweep the recomputation and the adjoint chain run at the same time
// and share the GPU, and in a batch all instances do: there the one-step pair timed side by side wins (two-step
// launches recompute a halo; on 512x256 (two-step, two-step) gave 13.0 and the side-by-side pair of 8-row tiles
// 15.0 G node-steps/s).  A binomial schedule whose slots hold every segment boundary is the sqrt layout and is
// pipelined the same way; other binomial and full-storage reverse sweeps run one chain and take the fastest variants.
// Explicit tile_rows fix all of them.
void choose_variants(lks_ctx* c) {
    if (c->prm.tile_rows != 0) {
        c->rows_fwd_sweep = c->eng->rows_f;
        c->rows_rec = c->prm.tile_rows_rec != 0 ? c->prm.tile_rows_rec : c->eng->rows_f;
        c->rows_adj = c->eng->rows_a;
    } else {
        const bool shared = c->throughput || c->pipelined;
        c->rows_fwd_sweep = c->throughput ? c->tune_f_one : c->tune_f_lat;
        c->rows_rec = shared ? c->tune_f_one : c->tune_f_lat;
        c->rows_adj = shared ? c->tune_a_one : c->tune_a_lat;
    }
    if (!c->eng->set_rows(c->rows_fwd_sweep, c->rows_adj, c->g) || !c->eng->set_rows(c->rows_rec, c->rows_adj, c->g))
        throw LksError{LKS_EINVAL, "step-kernel variant not available for this grid"};
    c->stats.tile_rows_fwd = c->rows_fwd_sweep;
    c->stats.tile_rows_rec = c->rows_rec;
    c->stats.tile_rows_adj = c->rows_adj;
}

void allocate(lks_ctx* c) {
    const lks_params& p = c->prm;
    const int D = c->D;
    const long long N = c->g.N;
    const size_t ts = c->tsize;
    c->state_bytes = (size_t)(D + 1) * N * ts;
    plan_checkpoints(c, c->state_bytes);
    {
        // the plan's large buffers (states, footprint-box records and factors, per-step slots) against the free
        // device memory, before any of them is allocated
        const long long S1 = (long long)c->S;
        const long long hist = p.ckpt == LKS_CKPT_FULL ? 0 : (c->pipelined ? 2 * S1 : S1);
        const long long states = (long long)c->slot_used.size() + hist + 7;
        const long long Lmax = c->Lmax, Fbn = c->g.Fbn;
        double need = (double)states * (double)c->state_bytes;
        need += (double)Lmax * Fbn * ts * (2.0 * 2 * D + 2 + (c->rot ? 1 + D : 1));  // box records, factors, kappa-bar
        need += (double)(p.Nt + 1) * (sizeof(Pose) + 8.0 * (4 * D + 2 * c->max_njb + 1));
        size_t free_b = 0, total_b = 0;
        LKS_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if (need > (double)free_b)
            throw LksError{LKS_ENOMEM, "the checkpoint and state plan needs " + std::to_string((long long)(need / 1e6)) +
                                           " MB of device memory, " + std::to_string((long long)(free_b / 1000000)) +
                                           " MB are free"};
    }

    c->d_gamma = (double*)dalloc(c, c->nd * 8);
    c->d_gt = (double*)dalloc(c, c->nd * 8);
    c->d_gb = (double*)dalloc(c, c->nd * 8);
    c->d_fnorm = (double*)dalloc(c, c->nd * 8);
    c->d_fscr = (double*)dalloc(c, c->nd * 8);
    c->d_tmp = (double*)dalloc(c, c->nd * 8);
    c->d_kref64 = (double*)dalloc(c, c->nde * 8);
    c->d_kref = dalloc(c, c->nde * ts);
    c->d_dkref = (double*)dalloc(c, c->nde * 8);
    c->d_knots = (double*)dalloc(c, (size_t)p.K * D * 8);
    c->d_filt = (double*)dalloc(c, (size_t)p.K * D * 8);
    c->d_ktmp = (double*)dalloc(c, (size_t)p.K * D * 8);
    c->d_tnorm = (double*)dalloc(c, (size_t)p.K * 8);
    c->d_s = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
    c->d_uG = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
    c->d_gs = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
    c->d_guG = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
    c->d_pose = (Pose*)dalloc(c, (size_t)(p.Nt + 1) * sizeof(Pose));
    // partials of n.u per step and probe block, then (with the variance term) their (n.u)^2 twins
    const long long nslot = (long long)(p.Nt + 1) * c->max_njb;
    c->g.jsq_off = p.phi_var != 0.0 ? nslot : 0;
    c->d_jslot = (double*)dalloc(c, (size_t)2 * nslot * 8);
    c->d_out_g = (double*)dalloc(c, c->nd * 8);
    c->d_out_k = (double*)dalloc(c, (size_t)p.K * D * 8);
    c->d_jstep = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
    c->d_J = (double*)dalloc(c, 4 * 8);  // J, E, V, 1 + 2 phi_var E
    c->g.obj = c->d_J;
    if (c->oar) {
        c->nbox = (int)nblk(c->g.Fbn, 256);
        const int onv = c->rot ? kOarRotNV : 2;  // per-step sums
        const long long ndb = nblk(c->nde, 256);
        // per-step sums only: the block partials of a launch live in scratch until its last block sums them
        c->d_oslot = (double*)dalloc(c, (size_t)(p.Nt + 1) * onv * 8);
        c->d_oms = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
        LKS_CUDA(cudaMemset(c->d_oms, 0, (size_t)(p.Nt + 1) * D * 8));
        c->d_oscr = (double*)dalloc(c, (size_t)std::max<long long>((long long)c->nbox * 2, c->rot ? ndb * onv : 0) * 8);
        if (c->rot) {
            c->d_okh = dalloc(c, (size_t)c->nde * ts);
            c->d_okl = dalloc(c, (size_t)c->nde * ts);
            c->d_ocst = (double*)dalloc(c, 4 * 8);
            c->d_ocscr = (double*)dalloc(c, (size_t)ndb * 4 * 8);
            c->d_oar_gth = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
            c->d_oar_gom = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
            LKS_CUDA(cudaMemset(c->d_oar_gth, 0, (size_t)(p.Nt + 1) * 8));
            LKS_CUDA(cudaMemset(c->d_oar_gom, 0, (size_t)(p.Nt + 1) * 8));
        }
        c->d_omsscr = (double*)dalloc(c, (size_t)c->Lmax * c->nbox * D * 8);
        c->d_otick = (unsigned*)dalloc(c, (size_t)(c->Lmax + 2) * sizeof(unsigned));
        LKS_CUDA(cudaMemset(c->d_otick, 0, (size_t)(c->Lmax + 2) * sizeof(unsigned)));
        c->d_oar_guG = (double*)dalloc(c, (size_t)(p.Nt + 1) * D * 8);
        c->d_oar_dK = (double*)dalloc(c, 8);
        LKS_CUDA(cudaMemset(c->d_oslot, 0, (size_t)(p.Nt + 1) * onv * 8));
        LKS_CUDA(cudaMemset(c->d_oar_guG, 0, (size_t)(p.Nt + 1) * D * 8));
    }
    c->d_flag = (unsigned*)dalloc(c, 16);  // [0] stability flag of the last forward, [1] status word (Geom::status)
    LKS_CUDA(cudaMemset(c->d_flag, 0, 16));
    c->g.status = c->d_flag + 1;
    // kappa-bar per step (and u^S-bar with a rotating body); per-block motion partials per step (2 D values, and
    // dJ/dtheta, dJ/domega with a rotating body)
    c->d_kbar = dalloc(c, (size_t)c->Lmax * c->g.Fbn * ts * (c->rot ? 1 + D : 1));
    c->nsb = c->rot ? (int)nblk(c->g.Fbn, 256) : c->eng->sens_blocks(c->g, c->alks);  // blocks per step of the sensitivities
    c->d_mslot = (double*)dalloc(c, (size_t)c->Lmax * c->nsb * (2 * D + (c->rot ? 2 : 0)) * 8);
    c->d_mpart = (double*)dalloc(c, (size_t)c->Lmax * kMotionChunks * (2 * D + (c->rot ? 2 : 0)) * 8);
    if (c->rot) {
        const int Kw = p.K_w;
        c->d_aknots = (double*)dalloc(c, (size_t)Kw * 8);
        c->d_afilt = (double*)dalloc(c, (size_t)Kw * 8);
        c->d_anorm = (double*)dalloc(c, (size_t)Kw * 8);
        c->d_atmp = (double*)dalloc(c, (size_t)Kw * 8);
        c->d_out_a = (double*)dalloc(c, (size_t)Kw * 8);
        c->d_theta = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
        c->d_omega = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
        c->d_gth = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
        c->d_gom = (double*)dalloc(c, (size_t)(p.Nt + 1) * 8);
        c->d_rotmap = dalloc(c, (size_t)(1 + D) * c->g.Fbn * ts);
        c->g.rotmap = c->d_rotmap;
        LKS_CUDA(cudaMemset(c->d_aknots, 0, (size_t)Kw * 8));
        LKS_CUDA(cudaMemset(c->d_out_a, 0, (size_t)Kw * 8));
        LKS_CUDA(cudaMemset(c->d_gth, 0, (size_t)(p.Nt + 1) * 8));
        LKS_CUDA(cudaMemset(c->d_gom, 0, (size_t)(p.Nt + 1) * 8));
        LKS_CUDA(cudaMemset(c->d_rotmap, 0, (size_t)(1 + D) * c->g.Fbn * ts));
    }
    c->box_step = 2LL * D * c->g.Fbn;
    c->d_boxbuf = dalloc(c, (size_t)2 * c->Lmax * c->box_step * ts);
    c->d_fac = dalloc(c, (size_t)2 * c->Lmax * c->g.Fbn * ts);
    LKS_CUDA(cudaMemset(c->d_fac, 0, (size_t)2 * c->Lmax * c->g.Fbn * ts));

    const size_t sb = c->state_bytes;
    c->slot.resize(c->slot_used.size());
    for (auto& s : c->slot) s = dalloc(c, sb);
    for (int h = 0; h < 2; ++h) {
        c->hist[h].assign(c->S + 1, nullptr);
        // the second buffer serves the pipelined sweep only
        if (p.ckpt != LKS_CKPT_FULL && (h == 0 || c->pipelined))
            for (int k = 1; k <= c->S; ++k) c->hist[h][k] = dalloc(c, sb);
    }
    c->pp[0] = dalloc(c, sb);
    c->pp[1] = dalloc(c, sb);
    c->pp[2] = dalloc(c, sb);
    c->tmp_state = dalloc(c, sb);
    c->fin = dalloc(c, sb);
    c->lam[0] = dalloc(c, sb);
    c->lam[1] = dalloc(c, sb);
    if (c->alks) {
        const size_t ab = (size_t)(1 + D + D * (D + 1) / 2) * N * ts;
        c->alam[0] = dalloc(c, ab);
        c->alam[1] = dalloc(c, ab);
    }
    c->stats.ckpt_slots = (int32_t)c->slot.size();
    c->stats.seg_len = c->S;
    c->stats.pipelined = c->pipelined ? 1 : 0;

    LKS_CUDA(cudaHostAlloc((void**)&c->h_flag, 16, cudaHostAllocDefault));
    std::memset(c->h_flag, 0, 16);
    LKS_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    LKS_CUDA(cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking));
    LKS_CUDA(cudaStreamCreateWithFlags(&c->cap3, cudaStreamNonBlocking));
    LKS_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    LKS_CUDA(cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        LKS_CUDA(cudaEventCreateWithFlags(&c->ev_rec[i], cudaEventDisableTiming));
        LKS_CUDA(cudaEventCreateWithFlags(&c->ev_adj[i], cudaEventDisableTiming));
        LKS_CUDA(cudaEventCreateWithFlags(&c->ev_sens[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < 3; ++i) LKS_CUDA(cudaEventCreateWithFlags(&c->ev_sync[i], cudaEventDisableTiming));
    LKS_CUDA(cudaEventCreateWithFlags(&c->ev_flag, cudaEventDisableTiming));
    LKS_CUDA(cudaMemset(c->d_jslot, 0, (size_t)2 * nslot * 8));
    LKS_CUDA(cudaMemset(c->d_J, 0, 4 * 8));
    LKS_CUDA(cudaMemset(c->d_pose, 0, (size_t)(p.Nt + 1) * sizeof(Pose)));
    filter_norm_kernel<<<nblk(c->nd, 128), 128, cone_table_bytes(c->dg.R)>>>(c->dg, c->d_fnorm);
    LKS_LAUNCHED();
    motion_norm_kernel<<<nblk(p.K, 128), 128>>>(c->mg, c->d_tnorm);
    LKS_LAUNCHED();
    if (c->rot) {
        motion_norm_kernel<<<nblk(p.K_w, 128), 128>>>(c->mgw, c->d_anorm);
        LKS_LAUNCHED();
    }
    LKS_CUDA(cudaDeviceSynchronize());
}

cudaEvent_t next_event(lks_ctx* c) {
    if (c->evnext == c->evpool.size()) return nullptr;  // pool exhausted: the span goes untimed
    return c->evpool[c->evnext++];
}

// Mark the start of a timed span of one kind (0 forward steps, 1 recompute, 2 adjoint steps).
cudaEvent_t span_begin(lks_ctx* c, cudaStream_t s) {
    if (!c->timing) return nullptr;
    cudaEvent_t e = next_event(c);
    if (e) LKS_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    return e;
}

void span_end(lks_ctx* c, int kind, cudaEvent_t e0, cudaStream_t s) {
    if (!c->timing || !e0) return;
    cudaEvent_t e1 = next_event(c);
    if (!e1) return;
    LKS_CUDA(cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal));
    c->spans.push_back({kind, {e0, e1}});
}

// Run `body(stream)` eagerly, or capture it once into a graph on the internal stream and replay it on s.
template <typename F>
void run_graph(lks_ctx* c, cudaGraphExec_t& gx, cudaStream_t s, F&& body) {
    if (!c->use_graphs) {
        body(s);
        return;
    }
    if (!gx) {
        LKS_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        try {
            body(c->cap);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->cap, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        cudaGraph_t g = nullptr;
        LKS_CUDA(cudaStreamEndCapture(c->cap, &g));
        cudaError_t e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        LKS_CUDA(e);
    }
    LKS_CUDA(cudaGraphLaunch(gx, s));
}

void drop_graphs(lks_ctx* c) {
    if (c->gx_fwd) cudaGraphExecDestroy(c->gx_fwd);
    if (c->gx_adj) cudaGraphExecDestroy(c->gx_adj);
    c->gx_fwd = c->gx_adj = nullptr;
    c->evnext = 0;
    c->spans_fwd.clear();
    c->spans_adj.clear();
}

void free_all(lks_ctx* c) {
    drop_graphs(c);
    for (cudaStream_t* st : {&c->cap, &c->cap2, &c->cap3, &c->side, &c->side2}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
    for (int i = 0; i < 2; ++i) {
        for (cudaEvent_t* e : {&c->ev_rec[i], &c->ev_adj[i], &c->ev_sens[i]}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
    }
    for (int i = 0; i < 3; ++i) {
        if (c->ev_sync[i]) cudaEventDestroy(c->ev_sync[i]);
        c->ev_sync[i] = nullptr;
    }
    for (auto e : c->evpool) cudaEventDestroy(e);
    c->evpool.clear();
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    if (c->h_flag) cudaFreeHost(c->h_flag);
    c->h_flag = nullptr;
    if (c->ev_flag) cudaEventDestroy(c->ev_flag);
    c->ev_flag = nullptr;
    if (c->ev_end) cudaEventDestroy(c->ev_end);
    c->ev_end = nullptr;
}

// ------------------------------------------------------------------------------------------------
// Forward and reverse sweeps
// ------------------------------------------------------------------------------------------------
void prepare_design_and_motion(lks_ctx* c, cudaStream_t s) {
    // a0: gamma -> gamma~ -> gamma-bar -> kappa^ref
    density_filter_kernel<<<nblk(c->nd, 128), 128, cone_table_bytes(c->dg.R), s>>>(c->dg, c->d_gamma, c->d_fnorm,
                                                                                c->d_gt, 0);
    LKS_LAUNCHED();
    c->eng->kappa_ref(c->dg, c->d_gt, c->d_gb, c->d_kref64, c->d_kref, s);
    // a1: knots -> filtered -> s_n, u^G_n -> per-step pose
    const int K = c->prm.K, D = c->D, Nt = c->prm.Nt;
    motion_filter_kernel<<<nblk((long long)K * D, 128), 128, 0, s>>>(c->mg, c->d_knots, c->d_tnorm, c->d_filt, 0);
    LKS_LAUNCHED();
    interp_kernel<<<nblk((long long)(Nt + 1) * D, 256), 256, 0, s>>>(c->mg, c->d_filt, c->d_s, c->d_uG);
    LKS_LAUNCHED();
    if (c->rot) {  // angle knots -> filtered -> theta_n, omega_n = theta_n - theta_{n-1} (Eqs. psi_filtered, theta, omega)
        motion_filter_kernel<<<nblk(c->prm.K_w, 128), 128, 0, s>>>(c->mgw, c->d_aknots, c->d_anorm, c->d_afilt, 0);
        LKS_LAUNCHED();
        interp_kernel<<<nblk(Nt + 1, 256), 256, 0, s>>>(c->mgw, c->d_afilt, c->d_theta, c->d_omega);
        LKS_LAUNCHED();
        c->launches += 2;
    }
    pose_kernel<<<nblk(Nt + 1, 128), 128, 0, s>>>(c->g, D, c->o0[0], c->o0[1], c->o0[2], c->cosine, Nt, c->d_s, c->d_uG,
                                                  c->rot ? c->d_theta : nullptr, c->rot ? c->d_omega : nullptr, c->rb,
                                                  c->d_pose);
    LKS_LAUNCHED();
    c->launches += 5;
}

void fwd_step(lks_ctx* c, int n, const void* in, void* out, bool objective, cudaStream_t s);

}  // namespace

// probe-block window of the forward kernel's objective slots
static void probe_blocks(const lks_ctx* c, int lo[3], int cnt[3]) {
    const int T[3] = {(int)c->eng->ftile.x, (int)c->eng->ftile.y, (int)c->eng->ftile.z};
    const int G[3] = {(int)c->eng->fgrid.x, (int)c->eng->fgrid.y, (int)c->eng->fgrid.z};
    for (int a = 0; a < 3; ++a) {
        if (a >= c->D) {
            lo[a] = 0;
            cnt[a] = 1;
            continue;
        }
        int b0 = c->g.probe_lo[a] / T[a];
        int b1 = (c->g.probe_hi[a] - 1) / T[a];
        b1 = std::min(b1, G[a] - 1);
        lo[a] = b0;
        cnt[a] = b1 - b0 + 1;
    }
}

namespace {

int njb_of(const lks_ctx* c) {
    int lo[3], cnt[3];
    probe_blocks(c, lo, cnt);
    return cnt[0] * cnt[1] * cnt[2];
}

// fac: where the forward kernel also writes 1 / (1 + kappa) of step n on the footprint box (nullptr: not wanted,
// or the kernel cannot)
void fwd_step(lks_ctx* c, int n, const void* in, void* out, bool objective, cudaStream_t s, void* fac = nullptr) {
    if (c->rot) {  // kappa and u^S of step n on the footprint box, read by the step kernel
        c->eng->rot_box_map(c->g, c->d_pose + n, c->d_kref, c->d_rotmap, s);
        c->launches++;
    }
    int lo[3], cnt[3];
    probe_blocks(c, lo, cnt);
    const int njb = cnt[0] * cnt[1] * cnt[2];
    c->eng->fac_out = fac;
    c->eng->fwd(c->g, in, out, c->d_kref, c->d_pose + n,
                objective ? c->d_jslot + (long long)n * njb : nullptr, c->d_flag, lo, cnt, s);
    c->eng->fac_out = nullptr;
    c->launches++;
}

// Two forward steps n, n+1 (or step n alone when out2 is null) in one fused launch.
void fwd_pair(lks_ctx* c, int n, const void* in, void* out1, void* out2, bool objective, cudaStream_t s) {
    int lo[3], cnt[3];
    probe_blocks(c, lo, cnt);
    const int njb = cnt[0] * cnt[1] * cnt[2];
    c->eng->fwd2(c->g, in, out1, out2, c->d_kref, c->d_pose + n, objective ? c->d_jslot + (long long)n * njb : nullptr,
                 objective && out2 ? c->d_jslot + (long long)(n + 1) * njb : nullptr, c->d_flag, lo, cnt, s);
    c->launches++;
}

// Objective J2: the footprint partials of state n (read before its buffer is reused, in stream order).
void oar_partial(lks_ctx* c, int n, const void* st, cudaStream_t s) {
    if (c->rot) {
        c->eng->oar_rot_partial(c->g, c->ogeo, c->d_pose + n, c->d_kref, st, c->d_okh, c->d_okl, c->d_oscr,
                                c->d_otick, c->d_oslot + (long long)kOarRotNV * n, s);
        c->launches++;
        return;
    }
    c->eng->oar_partial(c->g, c->d_pose + n, c->d_kref, st, c->d_oscr, c->d_otick, c->d_oslot + 2LL * n, s);
    c->launches++;
}

// Steps n0+1 .. n1 from the state at `in`; dst(n) names the buffer of state n (distinct from the state it is
// computed from).  Pairs of steps go to one fused launch when the forward kernel supports it.  fac_base: when set
// and the forward kernel writes them (Engine::fwd_writes_fac), the footprint-box factors 1 / (1 + kappa) of step n go
// to fac_base + (n - n0 - 1) Fbn elements.
template <typename Dst>
const void* run_steps(lks_ctx* c, int n0, int n1, const void* in, Dst&& dst, bool objective, cudaStream_t s,
                      void* fac_base = nullptr) {
    const void* cur = in;
    int n = n0 + 1;
    while (n <= n1) {
        if (c->eng->fused2()) {
            const bool two = n + 1 <= n1;
            void* o1 = dst(n);
            void* o2 = two ? dst(n + 1) : nullptr;
            fwd_pair(c, n, cur, o1, o2, objective, s);
            if (objective && c->oar) {
                oar_partial(c, n, o1, s);
                if (two) oar_partial(c, n + 1, o2, s);
            }
            cur = two ? o2 : o1;
            n += two ? 2 : 1;
        } else {
            void* o = dst(n);
            fwd_step(c, n, cur, o, objective, s,
                     fac_base != nullptr ? c->tptr(fac_base, (long long)(n - n0 - 1) * c->g.Fbn) : nullptr);
            if (objective && c->oar) oar_partial(c, n, o, s);
            cur = o;
            ++n;
        }
    }
    return cur;
}

// Round-robin over the three ping-pong buffers, never handing out `avoid` (the state being read).
struct PingPong {
    lks_ctx* c;
    int i = 0;
    void* next(const void* avoid) {
        for (int k = 0; k < 3; ++k) {
            void* p = c->pp[i];
            i = (i + 1) % 3;
            if (p != avoid) return p;
        }
        return nullptr;
    }
};

void forward_body(lks_ctx* c, cudaStream_t s);

void run_forward(lks_ctx* c, cudaStream_t s) {
    if (c->use_graphs && !c->gx_fwd) {
        // a new forward capture starts a new timing-event layout; the reverse sweep is re-captured after it
        drop_graphs(c);
    }
    run_graph(c, c->gx_fwd, s, [&](cudaStream_t cs) { forward_body(c, cs); });
    LKS_CUDA(cudaEventRecord(c->ev_flag, s));
    if (!c->use_graphs) c->spans_fwd = c->spans;
    c->stats.forward_steps = c->prm.Nt;
    c->have_forward = true;
    c->have_final = true;
}

void forward_body(lks_ctx* c, cudaStream_t s) {
    const int Nt = c->prm.Nt;
    c->eng->set_rows(c->rows_fwd_sweep, c->rows_adj, c->g);
    c->launches = 0;
    if (!c->use_graphs) c->evnext = 0;
    c->spans.clear();
    cudaEvent_t eall = span_begin(c, s);
    c->ev_all0 = eall;
    prepare_design_and_motion(c, s);
    LKS_CUDA(cudaMemsetAsync(c->d_flag, 0, 4, s));
    // boundary 0 lives in slot 0
    std::fill(c->slot_of.begin(), c->slot_of.end(), -1);
    std::fill(c->slot_used.begin(), c->slot_used.end(), 0);
    c->slot_of[0] = 0;
    c->slot_used[0] = 1;
    std::vector<char> store(c->M + 1, 0);
    if (c->prm.ckpt == LKS_CKPT_REVOLVE) {
        for (int m : c->chain) store[m] = 1;
    } else {
        for (int m = 1; m < c->M; ++m) store[m] = 1;
    }
    if (c->custom_init)
        LKS_CUDA(cudaMemcpyAsync(c->slot[0], c->d_init, c->state_bytes, cudaMemcpyDeviceToDevice, s));
    else
        c->eng->init_state(c->g, c->slot[0], s);
    c->launches++;
    if (c->oar && c->rot) {  // J2 with a rotating body: clear the per-node accumulation, K / M1 / I of kappa^ref
        LKS_CUDA(cudaMemsetAsync(c->d_okh, 0, (size_t)c->nde * c->tsize, s));
        LKS_CUDA(cudaMemsetAsync(c->d_okl, 0, (size_t)c->nde * c->tsize, s));
        oar_rot_const_kernel<<<nblk(c->nde, 256), 256, 0, s>>>(c->d_kref64, c->g.nde[0], c->g.nde[1], c->g.nde[2],
                                                               c->d_ocscr, c->d_otick + c->Lmax + 1, c->d_ocst);
        LKS_LAUNCHED();
        c->launches++;
    }
    PingPong pp{c};
    cudaEvent_t e0 = span_begin(c, s);
    // state n goes to the final buffer, its checkpoint slot, or a ping-pong buffer
    auto dst = [&](int n) -> void* {
        if (n == Nt) return c->fin;
        if (n % c->S == 0 && store[n / c->S]) {
            const int m = n / c->S;
            const int si = (int)(std::find(c->slot_used.begin(), c->slot_used.end(), 0) - c->slot_used.begin());
            if (si >= (int)c->slot.size()) throw LksError{LKS_ESTATE, "internal: out of checkpoint slots"};
            c->slot_used[si] = 1;
            c->slot_of[m] = si;
            return c->slot[si];
        }
        return pp.next(nullptr);
    };
    run_steps(c, 0, Nt, c->slot[0], dst, true, s);
    span_end(c, 0, e0, s);
    objective_reduce_kernel<<<1, 256, 0, s>>>(c->d_jslot, c->g.jsq_off, njb_of(c), Nt, c->g.phi, c->g.phi_var,
                                              c->d_jstep, c->d_J);
    LKS_LAUNCHED();
    c->launches++;
    if (c->oar && c->rot) {
        oar_rot_reduce_kernel<<<1, 256, 0, s>>>(c->ogeo, c->d_oslot, Nt, c->d_pose, c->d_ocst, c->D, c->d_J, c->d_oms,
                                                c->d_oar_guG, c->d_oar_gth, c->d_oar_gom);
        LKS_LAUNCHED();
        c->launches++;
    } else if (c->oar) {
        oar_reduce_kernel<<<1, 256, 0, s>>>(c->ogeo, c->d_oslot, Nt, c->d_pose, c->d_kref64, (long long)c->nde,
                                            c->D, c->d_J, c->d_oar_guG, c->d_oar_dK);
        LKS_LAUNCHED();
        c->launches++;
    }
    LKS_CUDA(cudaMemcpyAsync(c->h_flag, c->d_flag, 8, cudaMemcpyDeviceToHost, s));
    c->launches_fwd = c->launches;
    c->spans_fwd = c->spans;
}

// Advance from the state at step n0 (pointer in) to step n1, writing the final state to out (out != in).
void advance(lks_ctx* c, int n0, int n1, const void* in, void* out, cudaStream_t s) {
    cudaEvent_t e0 = span_begin(c, s);
    PingPong pp{c};
    auto dst = [&](int n) -> void* { return n == n1 ? out : pp.next(in); };
    run_steps(c, n0, n1, in, dst, false, s);
    c->stats.recompute_steps += n1 - n0;
    span_end(c, 1, e0, s);
}

// Rebuild the states a+1..b of a segment that are not stored (into history buffer `buf`) and record where
// every state a..b of the segment lives.
void recompute_segment(lks_ctx* c, int a, int b, const void* start, const void* end, int buf, cudaStream_t s) {
    const int L = b - a;
    std::vector<const void*>& st = c->seg_st[buf];
    st.assign(L + 1, nullptr);
    st[0] = start;
    const bool full = c->prm.ckpt == LKS_CKPT_FULL;
    c->fac_written[buf] = 0;
    cudaEvent_t er = full ? nullptr : span_begin(c, s);
    if (full) {
        for (int j = 1; j <= L; ++j) {
            const int m = a + j;  // every state is a stored boundary in FULL mode
            st[j] = (j == L && end != nullptr) ? end : (m == c->prm.Nt) ? c->fin : c->slot[c->slot_of[m]];
        }
    } else {
        // rebuild states a+1 .. last into the history (the segment end comes from its checkpoint when stored)
        const int last = end != nullptr ? L - 1 : L;
        for (int j = 1; j <= last; ++j) st[j] = c->hist[buf][j];
        if (end != nullptr) st[L] = end;
        if (last >= 1) {
            auto dst = [&](int n) -> void* { return c->hist[buf][n - a]; };
            // the recompute also writes the adjoint's factors of its steps when its kernel can (the rest come from
            // box_fac in adjoint_segment)
            const bool fac = c->eng->fwd_writes_fac() && !c->rot && !c->alks && !c->eng->fused2();
            run_steps(c, a, a + last, start, dst, false, s,
                      fac ? c->tptr(c->d_fac, (long long)buf * c->Lmax * c->g.Fbn) : nullptr);
            if (fac) c->fac_written[buf] = last;
            c->stats.recompute_steps += last;
        }
    }
    span_end(c, 1, er, s);
}

// Adjoint steps n = b..a+1 of a segment whose states were laid out by recompute_segment(buf); each step also
// records lam_u and u_n on the footprint box into box buffer `buf` for sens_segment.
void alks_launch(lks_ctx* c, bool init, const void* lam_in, void* lam_out, const void* cur, int n, void* boxbuf, int src,
                 cudaStream_t s);

void adjoint_segment(lks_ctx* c, int a, int b, int buf, cudaStream_t s) {
    const std::vector<const void*>& st = c->seg_st[buf];
    cudaEvent_t ea = span_begin(c, s);
    if (c->alks) {  // the ALKS: one step kernel per step, with the flow state of the same step
        for (int n = b; n > a; --n) {
            void* bb = c->tptr(c->d_boxbuf, ((long long)buf * c->Lmax + (n - a - 1)) * c->box_step);
            alks_launch(c, false, c->alam[0], c->alam[1], st[n - a], n, bb, n - 1 >= 1 ? 1 : 0, s);
            std::swap(c->alam[0], c->alam[1]);
            c->stats.adjoint_steps++;
            c->launches++;
        }
        span_end(c, 2, ea, s);
        return;
    }
    // 1 / (1 + kappa) on the footprint box for the steps of the segment that the recompute did not write (all of
    // them unless its kernel writes them), in one launch
    const int fw = c->fac_written[buf];
    if (c->rot) {
        c->eng->rot_box_fac(c->g, c->d_pose, c->d_kref, a + 1, b - a,
                            c->tptr(c->d_fac, (long long)buf * c->Lmax * c->g.Fbn), s);
        c->launches++;
    } else if (fw < b - a) {
        c->eng->box_fac(c->g, c->d_pose, c->d_kref, a + 1 + fw, b - a - fw,
                        c->tptr(c->d_fac, ((long long)buf * c->Lmax + fw) * c->g.Fbn), s);
        c->launches++;
    }
    for (int n = b; n > a;) {
        const int j = n - a - 1;  // box-buffer slot of step n
        void* bb = c->tptr(c->d_boxbuf, ((long long)buf * c->Lmax + j) * c->box_step);
        const void* fc = c->tptr(c->d_fac, ((long long)buf * c->Lmax + j) * c->g.Fbn);
        // J2 adds the source of step n to lambda_n before the step reads it, so its steps go one per launch
        if (c->oar) {
            if (c->rot)
                c->eng->oar_rot_source(c->g, c->ogeo, c->d_pose + n, c->d_kref, c->lam[0], s);
            else
                c->eng->oar_source(c->g, c->ogeo, c->d_pose + n, c->d_kref, c->lam[0], s);
            c->launches++;
        }
        if (c->eng->fused_adj2() && n - 1 > a && !c->oar) {  // steps n and n-1 in one launch
            void* bb2 = c->tptr(c->d_boxbuf, ((long long)buf * c->Lmax + j - 1) * c->box_step);
            const void* fc2 = c->tptr(c->d_fac, ((long long)buf * c->Lmax + j - 1) * c->g.Fbn);
            c->eng->adj2(c->g, c->lam[0], c->lam[1], st[n - 1 - a], st[n - a], st[n - 2 - a], c->d_kref,
                         c->d_pose + n, bb, fc, n - 1 >= 1 ? 1 : 0, bb2, fc2, n - 2 >= 1 ? 1 : 0, s);
            c->stats.adjoint_steps += 2;
            n -= 2;
        } else {
            c->eng->adj(c->g, c->lam[0], c->lam[1], st[n - 1 - a], st[n - a], c->d_kref, c->d_pose + n, bb, fc,
                        n - 1 >= 1 && !c->oar ? 1 : 0, s);
            c->stats.adjoint_steps++;
            n -= 1;
        }
        std::swap(c->lam[0], c->lam[1]);
        c->launches++;
    }
    span_end(c, 2, ea, s);
}

// Local sensitivities of a segment's steps from box buffer `buf`, folded into the design gradient (strict step
// order) and the per-step motion gradients.
void sens_segment(lks_ctx* c, int a, int b, int buf, cudaStream_t s) {
    const int L = b - a;
    const int mode = c->prm.mode;
    const bool shape = mode != LKS_MODE_MOTION, motion = mode != LKS_MODE_SHAPE;
    const void* bb = c->tptr(c->d_boxbuf, (long long)buf * c->Lmax * c->box_step);
    if (c->rot) {
        // rotating body: kappa-bar and u^S-bar per box node, the motion partials (position, u^G, theta, omega), the
        // transposed mapping on the design side, and the per-step motion sums
        const long long kst = (long long)(1 + c->D) * c->g.Fbn;
        c->eng->rot_sens(c->g, c->d_pose, c->d_kref, bb, c->box_step, a + 1, L, c->d_kbar, c->d_mslot, s);
        c->launches++;
        if (shape) {
            c->eng->rot_gather(c->g, c->d_pose, c->d_kbar, a + 1, L, kst, c->d_dkref, s);
            c->launches++;
        }
        if (motion) {
            const dim3 cg(L, kMotionChunks);
            if (c->D == 2) {
                motion_chunk_kernel<6><<<cg, 128, 0, s>>>(c->d_mslot, c->nsb, kMotionChunks, c->d_mpart);
                rot_motion_reduce_kernel<2><<<L, 32, 0, s>>>(c->d_mpart, kMotionChunks, a + 1, L, c->d_gs, c->d_guG,
                                                            c->d_gth, c->d_gom);
            } else {
                motion_chunk_kernel<8><<<cg, 128, 0, s>>>(c->d_mslot, c->nsb, kMotionChunks, c->d_mpart);
                rot_motion_reduce_kernel<3><<<L, 32, 0, s>>>(c->d_mpart, kMotionChunks, a + 1, L, c->d_gs, c->d_guG,
                                                            c->d_gth, c->d_gom);
            }
            LKS_LAUNCHED();
            c->launches += 2;
        }
        return;
    }
    c->eng->sens(c->g, c->d_pose, c->d_kref, bb, c->box_step, a + 1, L, shape ? c->d_kbar : nullptr,
                 motion ? c->d_mslot : nullptr, c->alks, s);
    c->launches++;
    if (c->oar) {
        c->eng->oar_sens(c->g, c->ogeo, c->d_pose, c->d_kref, bb, c->box_step, a + 1, L, shape ? c->d_kbar : nullptr,
                         c->d_omsscr, c->d_otick + 1, c->d_oms, s);
        c->launches++;
    }
    if (shape) {
        c->eng->gather(c->g, c->d_pose, c->d_kbar, a + 1, L, c->g.Fbn, c->d_dkref, s);
        c->launches++;
    }
    if (motion) {
        const dim3 cg(L, kMotionChunks);
        if (c->D == 2) {
            motion_chunk_kernel<4><<<cg, 128, 0, s>>>(c->d_mslot, c->nsb, kMotionChunks, c->d_mpart);
            motion_reduce_kernel<2><<<L, 32, 0, s>>>(c->d_mpart, kMotionChunks, a + 1, L, c->d_gs, c->d_guG);
        } else {
            motion_chunk_kernel<6><<<cg, 128, 0, s>>>(c->d_mslot, c->nsb, kMotionChunks, c->d_mpart);
            motion_reduce_kernel<3><<<L, 32, 0, s>>>(c->d_mpart, kMotionChunks, a + 1, L, c->d_gs, c->d_guG);
        }
        LKS_LAUNCHED();
        c->launches += 2;
    }
}

// Reverse one segment (steps a+1..b) on one stream.
void do_segment(lks_ctx* c, int a, int b, const void* start, const void* end, cudaStream_t s) {
    recompute_segment(c, a, b, start, end, 0, s);
    adjoint_segment(c, a, b, 0, s);
    sens_segment(c, a, b, 0, s);
}

// sqrt(N) reverse sweep as three concurrent chains: the recompute of segment m-1 (stream B) and the
// sensitivities of segment m+1 (stream C) overlap the adjoint steps of segment m (stream A).  History and box
// buffers are double-buffered; the events keep each buffer's producer and consumer in order.
void reverse_sqrt_pipelined(lks_ctx* c, cudaStream_t A, cudaStream_t B, cudaStream_t Cs) {
    LKS_CUDA(cudaEventRecord(c->ev_sync[0], A));
    LKS_CUDA(cudaStreamWaitEvent(B, c->ev_sync[0], 0));
    LKS_CUDA(cudaStreamWaitEvent(Cs, c->ev_sync[0], 0));
    int idx = 0;
    for (int m = c->M - 1; m >= 0; --m, ++idx) {
        const int buf = idx & 1;
        const int a = c->step_of(m), b = c->step_of(m + 1);
        if (idx >= 2) LKS_CUDA(cudaStreamWaitEvent(B, c->ev_adj[buf], 0));  // history buffer released
        recompute_segment(c, a, b, c->slot[c->slot_of[m]], m + 1 == c->M ? c->fin : c->slot[c->slot_of[m + 1]], buf, B);
        LKS_CUDA(cudaEventRecord(c->ev_rec[buf], B));
        LKS_CUDA(cudaStreamWaitEvent(A, c->ev_rec[buf], 0));
        if (idx >= 2) LKS_CUDA(cudaStreamWaitEvent(A, c->ev_sens[buf], 0));  // box buffer released
        adjoint_segment(c, a, b, buf, A);
        LKS_CUDA(cudaEventRecord(c->ev_adj[buf], A));
        LKS_CUDA(cudaStreamWaitEvent(Cs, c->ev_adj[buf], 0));
        sens_segment(c, a, b, buf, Cs);
        LKS_CUDA(cudaEventRecord(c->ev_sens[buf], Cs));
    }
    LKS_CUDA(cudaEventRecord(c->ev_sync[1], B));
    LKS_CUDA(cudaEventRecord(c->ev_sync[2], Cs));
    LKS_CUDA(cudaStreamWaitEvent(A, c->ev_sync[1], 0));
    LKS_CUDA(cudaStreamWaitEvent(A, c->ev_sync[2], 0));
}

int take_slot(lks_ctx* c) {
    for (size_t i = 0; i < c->slot_used.size(); ++i)
        if (!c->slot_used[i]) {
            c->slot_used[i] = 1;
            return (int)i;
        }
    throw LksError{LKS_ESTATE, "internal: out of checkpoint slots"};
}

// Binomial reverse sweep over segments [ma, mb) with the state of boundary ma at `ap` and `freec` free slots.
void reverse_revolve(lks_ctx* c, int ma, int mb, int freec, const void* ap, cudaStream_t s) {
    const int a = c->step_of(ma);
    if (mb - ma == 1) {
        do_segment(c, a, c->step_of(mb), ap, mb == c->M ? c->fin : nullptr, s);
        return;
    }
    if (freec == 0) {
        for (int m = mb - 1; m >= ma; --m) {
            const void* sp = ap;
            if (m > ma) {
                advance(c, a, c->step_of(m), ap, c->tmp_state, s);
                sp = c->tmp_state;
            }
            do_segment(c, c->step_of(m), c->step_of(m + 1), sp, m + 1 == c->M ? c->fin : nullptr, s);
        }
        return;
    }
    const int mm = ma + binom_split(mb - ma, freec);
    int si = c->slot_of[mm];
    if (si < 0) {
        si = take_slot(c);
        c->slot_of[mm] = si;
        advance(c, a, c->step_of(mm), ap, c->slot[si], s);
    }
    reverse_revolve(c, mm, mb, freec - 1, c->slot[si], s);
    c->slot_used[si] = 0;
    c->slot_of[mm] = -1;
    reverse_revolve(c, ma, mm, freec, ap, s);
}

void adjoint_body(lks_ctx* c, cudaStream_t s);

void run_adjoint(lks_ctx* c, cudaStream_t s) {
    if (!c->have_forward) throw LksError{LKS_ESTATE, "lks_adjoint needs a preceding lks_forward"};
    // no wait for the forward's stability flag here: the reverse sweep is enqueued behind it, and an unstable forward
    // is reported by lks_get_status, by lks_adjoint (host pointers) and as NaN gradients of lks_adjoint_dev
    run_graph(c, c->gx_adj, s, [&](cudaStream_t cs) { adjoint_body(c, cs); });
    c->have_lambda0 = !c->alks;  // the ALKS state at n = 0 is not the gradient with respect to the initial state
    if (!c->use_graphs) c->spans_adj = c->spans;
    // the binomial schedule reuses the forward's checkpoint slots: a new forward must precede the next adjoint
    if (c->prm.ckpt == LKS_CKPT_REVOLVE) c->have_forward = false;
}

void adjoint_body(lks_ctx* c, cudaStream_t s) {
    const int Nt = c->prm.Nt, D = c->D, K = c->prm.K;
    c->eng->set_rows(c->rows_rec, c->rows_adj, c->g);
    c->launches = 0;
    c->spans.clear();
    c->stats.recompute_steps = 0;
    c->stats.adjoint_steps = 0;
    LKS_CUDA(cudaMemsetAsync(c->d_dkref, 0, c->nde * 8, s));
    LKS_CUDA(cudaMemsetAsync(c->d_gs, 0, (size_t)(Nt + 1) * D * 8, s));
    LKS_CUDA(cudaMemsetAsync(c->d_guG, 0, (size_t)(Nt + 1) * D * 8, s));
    if (c->rot) {
        LKS_CUDA(cudaMemsetAsync(c->d_gth, 0, (size_t)(Nt + 1) * 8, s));
        LKS_CUDA(cudaMemsetAsync(c->d_gom, 0, (size_t)(Nt + 1) * 8, s));
    }
    if (c->alks)
        alks_launch(c, true, nullptr, c->alam[0], nullptr, Nt, nullptr, 1, s);
    else
        c->eng->init_adjoint(c->g, c->fin, c->lam[0], c->oar ? 0 : 1, s);
    c->launches++;
    if (c->custom_lterm) {  // the adjoint half of the periodic approximation (Sec. 3.3)
        c->eng->add_state(c->g, c->lam[0], c->d_lterm, s);
        c->launches++;
    }
    if (c->prm.ckpt == LKS_CKPT_REVOLVE && !c->pipelined) {
        reverse_revolve(c, 0, c->M, c->free_slots, c->slot[0], s);
    } else if (c->prm.ckpt == LKS_CKPT_FULL) {
        for (int b = Nt; b > 0; b -= c->Lmax) {
            const int a = std::max(0, b - c->Lmax);
            do_segment(c, a, b, a == 0 ? c->slot[0] : c->slot[c->slot_of[a]], b == Nt ? c->fin : c->slot[c->slot_of[b]], s);
        }
    } else {
        const bool cap = s == c->cap;
        reverse_sqrt_pipelined(c, s, cap ? c->cap2 : c->side, cap ? c->cap3 : c->side2);
    }
    if (c->oar) {  // J2's position terms and its explicit dependences on u^G and kappa^ref (and theta, omega)
        const long long nmax = std::max<long long>((long long)c->nde, (long long)Nt + 1);
        if (c->rot && c->tsize == 4)
            oar_rot_apply_kernel<float><<<nblk(nmax, 256), 256, 0, s>>>(
                Nt, D, c->d_oms, c->d_oar_guG, c->d_oar_gth, c->d_oar_gom, (const float*)c->d_okh,
                (const float*)c->d_okl, c->d_gs, c->d_guG, c->d_gth, c->d_gom, c->d_dkref, (long long)c->nde);
        else if (c->rot)
            oar_rot_apply_kernel<double><<<nblk(nmax, 256), 256, 0, s>>>(
                Nt, D, c->d_oms, c->d_oar_guG, c->d_oar_gth, c->d_oar_gom, (const double*)c->d_okh,
                (const double*)c->d_okl, c->d_gs, c->d_guG, c->d_gth, c->d_gom, c->d_dkref, (long long)c->nde);
        else
            oar_apply_kernel<<<nblk(nmax, 256), 256, 0, s>>>(Nt, D, c->d_oms, c->d_oar_guG, c->d_gs, c->d_guG,
                                                             c->d_oar_dK, c->d_dkref, (long long)c->nde);
        LKS_LAUNCHED();
        c->launches++;
    }
    // b6: chain rules
    design_chain_kernel<<<nblk(c->nd, 128), 128, 0, s>>>(c->dg, c->d_dkref, c->d_gt, c->d_gb, c->d_tmp);
    LKS_LAUNCHED();
    interp_T_kernel<<<nblk((long long)K * D, 64), 64, 0, s>>>(c->mg, c->d_gs, c->d_guG, c->d_ktmp);
    LKS_LAUNCHED();
    c->launches += 2;
    if (c->rot) {  // (dJ/dtheta_n, dJ/domega_n) -> difference^T, interpolation^T, filter^T -> dJ/d(angle knots)
        const int Kw = c->prm.K_w;
        if (c->prm.mode == LKS_MODE_SHAPE) {
            LKS_CUDA(cudaMemsetAsync(c->d_out_a, 0, (size_t)Kw * 8, s));
        } else {
            interp_T_kernel<<<nblk(Kw, 64), 64, 0, s>>>(c->mgw, c->d_gth, c->d_gom, c->d_atmp);
            LKS_LAUNCHED();
            motion_filter_kernel<<<nblk(Kw, 64), 64, 0, s>>>(c->mgw, c->d_atmp, c->d_anorm, c->d_out_a, 1);
            LKS_LAUNCHED();
            c->launches += 2;
        }
    }
    c->launches_adj = c->launches;
    c->spans_adj = c->spans;
    (void)K;
}

// Transposed density filter: in / norm into the context's scratch, then the weighted sums (identity for R <= 1).
void filter_T(lks_ctx* c, const double* in, double* out, cudaStream_t s) {
    const double* src = in;
    if (c->dg.R > 1.0) {
        filter_scale_kernel<<<nblk(c->nd, 256), 256, 0, s>>>(c->nd, in, c->d_fnorm, c->d_fscr);
        LKS_LAUNCHED();
        src = c->d_fscr;
    }
    density_filter_kernel<<<nblk(c->nd, 128), 128, cone_table_bytes(c->dg.R), s>>>(c->dg, src, c->d_fnorm, out, 1);
    LKS_LAUNCHED();
}

// Final gradients into caller buffers (device pointers), honouring the gradient mode.
void finish_adjoint(lks_ctx* c, double* dgamma, double* dpos, cudaStream_t s) {
    const int K = c->prm.K, D = c->D;
    c->launches = 0;
    if (dgamma) {
        if (c->prm.mode == LKS_MODE_MOTION) {
            LKS_CUDA(cudaMemsetAsync(dgamma, 0, c->nd * 8, s));
        } else {
            filter_T(c, c->d_tmp, dgamma, s);
            c->launches += 2;
        }
    }
    if (dpos) {
        if (c->prm.mode == LKS_MODE_SHAPE) {
            LKS_CUDA(cudaMemsetAsync(dpos, 0, (size_t)K * D * 8, s));
        } else {
            motion_filter_kernel<<<nblk((long long)K * D, 64), 64, 0, s>>>(c->mg, c->d_ktmp, c->d_tnorm, dpos, 1);
            LKS_LAUNCHED();
            c->launches++;
        }
    }
    c->stats.kernel_launches = c->launches_fwd + c->launches_adj + c->launches;
    if (c->timing && c->ev_all0 && c->ev_end) {
        LKS_CUDA(cudaEventRecord(c->ev_end, s));
        LKS_CUDA(cudaEventSynchronize(c->ev_end));
        double acc[3] = {0, 0, 0};
        for (auto* v : {&c->spans_fwd, &c->spans_adj})
            for (auto& sp : *v) {
                float ms = 0.f;
                LKS_CUDA(cudaEventElapsedTime(&ms, sp.second.first, sp.second.second));
                acc[sp.first] += ms;
            }
        float tot = 0.f;
        LKS_CUDA(cudaEventElapsedTime(&tot, c->ev_all0, c->ev_end));
        c->stats.ms_forward_steps = acc[0];
        c->stats.ms_recompute_steps = acc[1];
        c->stats.ms_adjoint_steps = acc[2];
        c->stats.ms_total = tot;
    }
}

// Arguments of the ALKS kernels in the engine's state precision (lam_in, lam_out: ALKS states; cur: flow state n).
template <typename T>
AlksArgs<T> make_alks_args(const lks_ctx* c, const void* lam_in, void* lam_out, const void* cur, int n, void* boxbuf,
                           int src) {
    AlksArgs<T> a;
    a.lam_in = (const T*)lam_in;
    a.lam_out = (T*)lam_out;
    a.u_cur = cur ? (const T*)cur + c->g.N : nullptr;
    a.kref = (const T*)c->d_kref;
    a.pose_n = c->d_pose + n;
    a.pose_m = c->d_pose + (n > 0 ? n - 1 : 0);
    a.boxbuf = (T*)boxbuf;
    a.src = src;
    for (int i = 0; i < 3; ++i) a.phi_dir3[i] = (T)(c->g.dir[i] * c->g.phi / 3.0);
    return a;
}

void alks_launch(lks_ctx* c, bool init, const void* lam_in, void* lam_out, const void* cur, int n, void* boxbuf, int src,
                 cudaStream_t s) {
    if (c->tsize == 4) {
        const AlksArgs<float> a = make_alks_args<float>(c, lam_in, lam_out, cur, n, boxbuf, src);
        if (init) c->eng->alks_init(c->g, c->d_pose + n, c->d_kref, lam_out, &a, s);
        else c->eng->alks_step(c->g, &a, s);
    } else {
        const AlksArgs<double> a = make_alks_args<double>(c, lam_in, lam_out, cur, n, boxbuf, src);
        if (init) c->eng->alks_init(c->g, c->d_pose + n, c->d_kref, lam_out, &a, s);
        else c->eng->alks_step(c->g, &a, s);
    }
}

// Errors that the device reports through the context's flag words (copied to h_flag by the calls that read them):
// an expired bounded wait (status word) first, as the cause of anything else, then the forward's stability flag.
void check_flags(lks_ctx* c) {
    if (c->h_flag[1] != 0u) throw LksError{LKS_ETIMEOUT, "a bounded device-side wait expired (tensor copies did not complete)"};
    if (c->h_flag[0] != 0u) throw LksError{LKS_EUNSTABLE, "forward sweep unstable: non-finite velocity or |u| > u_crit"};
}

// NaN gradients on the device when the last forward raised the stability flag or a bounded wait expired
// (asynchronous adjoint variants).
void poison_if_unstable(lks_ctx* c, double* dgamma, double* dpos, cudaStream_t s) {
    const long long nk = (long long)c->prm.K * c->D;
    const long long n = std::max<long long>(c->nd, nk);
    poison_unstable_kernel<<<nblk(n, 256), 256, 0, s>>>(c->d_flag, dgamma, c->nd, dpos, nk);
    LKS_LAUNCHED();
}

template <typename F>
int guard(lks_ctx* c, F&& f) {
    try {
        f();
        return LKS_OK;
    } catch (const LksError& e) {
        set_err(c, e);
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return LKS_ENOMEM;
    } catch (...) {
        if (c) c->err = "unexpected exception";
        return LKS_ECUDA;
    }
}

thread_local std::string g_create_err;

}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
// Host-pointer variants of the filter calls: the same kernels on device copies made for the call (allocated and
// freed here, on the legacy default stream), synchronous.
namespace {
struct DevScratch {
    double* p = nullptr;
    ~DevScratch() {
        if (p) cudaFree(p);
    }
};
// ins / outs: host arrays and their lengths; dev(inputs..., outputs...) runs the device variant on stream 0
template <typename F>
void host_roundtrip(std::initializer_list<std::pair<const double*, size_t>> ins,
                    std::initializer_list<std::pair<double*, size_t>> outs, F&& dev) {
    size_t total = 0;
    for (const auto& a : ins) {
        if (!a.first) throw LksError{LKS_EINVAL, "null pointer"};
        total += a.second;
    }
    for (const auto& a : outs) {
        if (!a.first) throw LksError{LKS_EINVAL, "null pointer"};
        total += a.second;
    }
    DevScratch b;
    LKS_CUDA(cudaMalloc(&b.p, std::max<size_t>(total, 1) * 8));
    std::vector<double*> d;
    double* q = b.p;
    for (const auto& a : ins) {
        LKS_CUDA(cudaMemcpy(q, a.first, a.second * 8, cudaMemcpyHostToDevice));
        d.push_back(q);
        q += a.second;
    }
    for (const auto& a : outs) {
        d.push_back(q);
        q += a.second;
    }
    const int rc = dev(d);
    if (rc != LKS_OK) throw LksError{rc, "device call failed"};
    size_t k = ins.size();
    for (const auto& a : outs) LKS_CUDA(cudaMemcpy(a.first, d[k++], a.second * 8, cudaMemcpyDeviceToHost));
}
}  // namespace

extern "C" {

int lks_default_params(lks_params* p) {
    if (!p) return LKS_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->size = sizeof(lks_params);
    p->lattice = LKS_D2Q9;
    p->n[0] = 64;
    p->n[1] = 32;
    p->n[2] = 1;
    p->periodic[0] = 1;
    p->periodic[1] = 0;
    p->periodic[2] = 1;
    p->nu = 0.02;
    p->kappa_max = 1.0;
    p->q = 0.1;
    p->nd[0] = 8;
    p->nd[1] = 8;
    p->nd[2] = 1;
    p->margin = 2;
    p->map_kernel = LKS_MAP_LINEAR;
    for (int a = 0; a < 3; ++a) p->base_center[a] = std::nan("");
    p->probe_lo[0] = 40;
    p->probe_lo[1] = 8;
    p->probe_lo[2] = 0;
    p->probe_hi[0] = 56;
    p->probe_hi[1] = 24;
    p->probe_hi[2] = 1;
    p->direction[0] = 1.0;
    p->Nt = 100;
    p->K = 10;
    p->R_t = 25.0;
    p->filter_R = 0.0;
    p->beta = 0.0;
    p->eta = 0.5;
    p->precision = LKS_FP64;
    p->ckpt = LKS_CKPT_FULL;
    p->mode = LKS_MODE_JOINT;
    p->u_crit = 0.3;
    p->l_m = 1.0;
    return LKS_OK;
}

const char* lks_strerror(int status) {
    switch (status) {
        case LKS_OK: return "ok";
        case LKS_EINVAL: return "invalid argument";
        case LKS_ENOMEM: return "out of memory";
        case LKS_ECUDA: return "CUDA error";
        case LKS_ESTATE: return "call order violated";
        case LKS_EUNSTABLE: return "unstable forward sweep";
        case LKS_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* lks_last_error_string(const lks_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

// A context; `throughput` (instances of a batch, which run concurrently) keeps the autotuner to variants that
// take one step per launch: the two-step variants shorten a lone instance's critical path by recomputing a
// halo, which costs throughput once many instances fill the GPU.
static int create_ctx(const lks_params* p, bool throughput, lks_ctx** out) {
    if (!out) return LKS_EINVAL;
    lks_ctx* c = nullptr;
    try {
        validate(p);
        c = new lks_ctx();
        c->prm = *p;
        c->throughput = throughput;
        std::memset(&c->stats, 0, sizeof(c->stats));
        setup_geometry(c);
        int ndev = 0;
        LKS_CUDA(cudaGetDeviceCount(&ndev));
        c->eng.reset(make_engine(p->precision, c->D, c->hw, c->g));
        choose_rows_initial(c);
        allocate(c);
        if (p->tile_rows == 0) autotune_rows(c);
        choose_variants(c);
        *out = c;
        g_create_err.clear();
        return LKS_OK;
    } catch (const LksError& e) {
        g_create_err = e.msg;
        if (c) {
            free_all(c);
            delete c;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        g_create_err = "host allocation failed";
        if (c) {
            free_all(c);
            delete c;
        }
        return LKS_ENOMEM;
    }
}

int lks_create(const lks_params* p, lks_ctx** out) { return create_ctx(p, false, out); }

void lks_destroy(lks_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
}

int lks_forward_dev(lks_ctx* c, const double* d_gamma, const double* d_pos, double* d_J, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!d_gamma || !d_pos) throw LksError{LKS_EINVAL, "null input pointer"};
        cudaStream_t s = (cudaStream_t)stream;
        LKS_CUDA(cudaMemcpyAsync(c->d_gamma, d_gamma, c->nd * 8, cudaMemcpyDeviceToDevice, s));
        LKS_CUDA(cudaMemcpyAsync(c->d_knots, d_pos, (size_t)c->prm.K * c->D * 8, cudaMemcpyDeviceToDevice, s));
        c->have_forward = c->have_final = false;
        run_forward(c, s);
        if (d_J) LKS_CUDA(cudaMemcpyAsync(d_J, c->d_J, 8, cudaMemcpyDeviceToDevice, s));
    });
}

int lks_forward(lks_ctx* c, const double* gamma, const double* pos, double* J) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!gamma || !pos || !J) throw LksError{LKS_EINVAL, "null pointer"};
        cudaStream_t s = 0;
        LKS_CUDA(cudaMemcpyAsync(c->d_gamma, gamma, c->nd * 8, cudaMemcpyHostToDevice, s));
        LKS_CUDA(cudaMemcpyAsync(c->d_knots, pos, (size_t)c->prm.K * c->D * 8, cudaMemcpyHostToDevice, s));
        c->have_forward = c->have_final = false;
        run_forward(c, s);
        double j = 0.0;
        LKS_CUDA(cudaMemcpyAsync(&j, c->d_J, 8, cudaMemcpyDeviceToHost, s));
        LKS_CUDA(cudaStreamSynchronize(s));
        check_flags(c);
        *J = j;
    });
}

int lks_adjoint_dev(lks_ctx* c, double* d_dgamma, double* d_dpos, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        run_adjoint(c, s);
        finish_adjoint(c, d_dgamma, d_dpos, s);
        poison_if_unstable(c, d_dgamma, d_dpos, s);
    });
}

int lks_adjoint(lks_ctx* c, double* dgamma, double* dpos) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!dgamma || !dpos) throw LksError{LKS_EINVAL, "null pointer"};
        cudaStream_t s = 0;
        run_adjoint(c, s);
        finish_adjoint(c, c->d_out_g, c->d_out_k, s);
        // the forward's flag reached the host before its sweep ended; the status word is read after the sweep
        LKS_CUDA(cudaMemcpyAsync(c->h_flag + 1, c->d_flag + 1, 4, cudaMemcpyDeviceToHost, s));
        LKS_CUDA(cudaStreamSynchronize(s));
        check_flags(c);
        LKS_CUDA(cudaMemcpyAsync(dgamma, c->d_out_g, c->nd * 8, cudaMemcpyDeviceToHost, s));
        LKS_CUDA(cudaMemcpyAsync(dpos, c->d_out_k, (size_t)c->prm.K * c->D * 8, cudaMemcpyDeviceToHost, s));
        LKS_CUDA(cudaStreamSynchronize(s));
    });
}

int lks_density_filter_dev(lks_ctx* c, const double* in, double* out, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!in || !out) throw LksError{LKS_EINVAL, "null pointer"};
        density_filter_kernel<<<nblk(c->nd, 128), 128, cone_table_bytes(c->dg.R), (cudaStream_t)stream>>>(
            c->dg, in, c->d_fnorm, out, 0);
        LKS_LAUNCHED();
    });
}

int lks_density_filter_T_dev(lks_ctx* c, const double* in, double* out, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!in || !out) throw LksError{LKS_EINVAL, "null pointer"};
        filter_T(c, in, out, (cudaStream_t)stream);
    });
}

int lks_gradient_step_dev(int64_t count, double step, const double* g, double* x, double lo, double hi, void* stream) {
    if (count < 0 || !g || !x || !(lo <= hi) || !std::isfinite(step)) return LKS_EINVAL;
    if (count == 0) return LKS_OK;
    gradient_step_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(count, step, g, x, lo, hi);
    return cudaGetLastError() == cudaSuccess ? LKS_OK : LKS_ECUDA;
}

int lks_projection_dev(int64_t count, double beta, double eta, const double* in, double* out, double* dout,
                       void* stream) {
    if (count < 0 || !in || !(beta >= 0.0) || !(eta > 0.0 && eta < 1.0)) return LKS_EINVAL;
    if (count == 0) return LKS_OK;
    projection_kernel<<<nblk(count, 256), 256, 0, (cudaStream_t)stream>>>(count, beta, eta, in, out, dout);
    return cudaGetLastError() == cudaSuccess ? LKS_OK : LKS_ECUDA;
}

int lks_motion_filter_dev(lks_ctx* c, const double* in, double* out, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!in || !out) throw LksError{LKS_EINVAL, "null pointer"};
        motion_filter_kernel<<<nblk((long long)c->prm.K * c->D, 64), 64, 0, (cudaStream_t)stream>>>(c->mg, in, c->d_tnorm, out, 0);
        LKS_LAUNCHED();
    });
}

int lks_motion_filter_T_dev(lks_ctx* c, const double* in, double* out, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!in || !out) throw LksError{LKS_EINVAL, "null pointer"};
        motion_filter_kernel<<<nblk((long long)c->prm.K * c->D, 64), 64, 0, (cudaStream_t)stream>>>(c->mg, in, c->d_tnorm, out, 1);
        LKS_LAUNCHED();
    });
}

int lks_interp_positions_dev(lks_ctx* c, const double* filt, double* s_out, double* uG, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!filt || !s_out || !uG) throw LksError{LKS_EINVAL, "null pointer"};
        interp_kernel<<<nblk((long long)(c->prm.Nt + 1) * c->D, 256), 256, 0, (cudaStream_t)stream>>>(c->mg, filt, s_out, uG);
        LKS_LAUNCHED();
    });
}

int lks_interp_positions_T_dev(lks_ctx* c, const double* gs, const double* guG, double* out, void* stream) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!gs || !guG || !out) throw LksError{LKS_EINVAL, "null pointer"};
        interp_T_kernel<<<nblk((long long)c->prm.K * c->D, 64), 64, 0, (cudaStream_t)stream>>>(c->mg, gs, guG, out);
        LKS_LAUNCHED();
    });
}


int lks_density_filter(lks_ctx* c, const double* in, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        host_roundtrip({{in, (size_t)c->nd}}, {{out, (size_t)c->nd}},
                       [&](std::vector<double*>& d) { return lks_density_filter_dev(c, d[0], d[1], nullptr); });
    });
}

int lks_density_filter_T(lks_ctx* c, const double* in, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        host_roundtrip({{in, (size_t)c->nd}}, {{out, (size_t)c->nd}},
                       [&](std::vector<double*>& d) { return lks_density_filter_T_dev(c, d[0], d[1], nullptr); });
    });
}

int lks_projection(int64_t count, double beta, double eta, const double* in, double* out, double* dout) {
    if (count < 0 || !in || (!out && !dout)) return LKS_EINVAL;
    if (count == 0) return LKS_OK;
    try {
        std::vector<double> unused;
        double* o = out;
        double* od = dout;
        if (!o) {
            unused.resize(count);
            o = unused.data();
        }
        if (!od) {
            if (unused.empty()) unused.resize(count);
            od = unused.data();
        }
        host_roundtrip({{in, (size_t)count}}, {{o, (size_t)count}, {od, (size_t)count}}, [&](std::vector<double*>& d) {
            return lks_projection_dev(count, beta, eta, d[0], d[1], d[2], nullptr);
        });
        return LKS_OK;
    } catch (const LksError& e) {
        return e.code;
    } catch (...) {
        return LKS_ENOMEM;
    }
}

int lks_motion_filter(lks_ctx* c, const double* knots, double* filtered) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        const size_t n = (size_t)c->prm.K * c->D;
        host_roundtrip({{knots, n}}, {{filtered, n}},
                       [&](std::vector<double*>& d) { return lks_motion_filter_dev(c, d[0], d[1], nullptr); });
    });
}

int lks_motion_filter_T(lks_ctx* c, const double* in, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        const size_t n = (size_t)c->prm.K * c->D;
        host_roundtrip({{in, n}}, {{out, n}},
                       [&](std::vector<double*>& d) { return lks_motion_filter_T_dev(c, d[0], d[1], nullptr); });
    });
}

int lks_interp_positions(lks_ctx* c, const double* filtered, double* s, double* uG) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        const size_t nk = (size_t)c->prm.K * c->D, ns = (size_t)(c->prm.Nt + 1) * c->D;
        host_roundtrip({{filtered, nk}}, {{s, ns}, {uG, ns}},
                       [&](std::vector<double*>& d) { return lks_interp_positions_dev(c, d[0], d[1], d[2], nullptr); });
    });
}

int lks_interp_positions_T(lks_ctx* c, const double* gs, const double* guG, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        const size_t nk = (size_t)c->prm.K * c->D, ns = (size_t)(c->prm.Nt + 1) * c->D;
        host_roundtrip({{gs, ns}, {guG, ns}}, {{out, nk}}, [&](std::vector<double*>& d) {
            return lks_interp_positions_T_dev(c, d[0], d[1], d[2], nullptr);
        });
    });
}

int lks_get_state(lks_ctx* c, double* p, double* u) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!p || !u) throw LksError{LKS_EINVAL, "null pointer"};
        if (!c->have_final) throw LksError{LKS_ESTATE, "no forward has run"};
        const long long N = c->g.N;
        double* dp = nullptr;
        LKS_CUDA(cudaMalloc(&dp, (size_t)(c->D + 1) * N * 8));
        c->eng->export_state(c->g, c->fin, dp, dp + N, 1.0 / 3.0, 0);
        cudaError_t e1 = cudaMemcpy(p, dp, N * 8, cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaMemcpy(u, dp + N, (size_t)c->D * N * 8, cudaMemcpyDeviceToHost);
        cudaFree(dp);
        LKS_CUDA(e1);
        LKS_CUDA(e2);
    });
}

int lks_get_step_sensitivities(lks_ctx* c, double* gs, double* guG) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!gs || !guG) throw LksError{LKS_EINVAL, "null pointer"};
        const size_t b = (size_t)(c->prm.Nt + 1) * c->D * 8;
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(gs, c->d_gs, b, cudaMemcpyDeviceToHost));
        LKS_CUDA(cudaMemcpy(guG, c->d_guG, b, cudaMemcpyDeviceToHost));
    });
}

int lks_get_objective_terms(lks_ctx* c, double* E, double* V) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!E || !V) throw LksError{LKS_EINVAL, "null pointer"};
        if (c->stats.forward_steps == 0) throw LksError{LKS_ESTATE, "no forward has run"};
        double t[4];
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(t, c->d_J, sizeof(t), cudaMemcpyDeviceToHost));
        *E = t[1];
        *V = t[2];
    });
}

int lks_set_timing(lks_ctx* c, int enable) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        const bool on = enable != 0;
        if (on == c->timing) return;
        drop_graphs(c);
        c->timing = on;
        if (on && c->evpool.empty()) {
            // two events per span: the forward sweep, and per segment a recompute and an adjoint span,
            // plus binomial-schedule advances
            const size_t need = 16 * (size_t)(c->M + 8) + 64;
            for (size_t i = 0; i < need; ++i) {
                cudaEvent_t e;
                LKS_CUDA(cudaEventCreate(&e));
                c->evpool.push_back(e);
            }
            LKS_CUDA(cudaEventCreate(&c->ev_end));
        }
    });
}

int lks_set_initial_state(lks_ctx* c, const double* p, const double* u) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if ((p == nullptr) != (u == nullptr)) throw LksError{LKS_EINVAL, "p and u must both be given or both NULL"};
        drop_graphs(c);  // the captured forward starts from the previous initial state
        c->have_forward = false;
        if (!p) {
            c->custom_init = false;
            return;
        }
        const long long N = c->g.N;
        if (!c->d_init) c->d_init = dalloc(c, c->state_bytes);
        DevScratch b;
        LKS_CUDA(cudaMalloc(&b.p, (size_t)(c->D + 1) * N * 8));
        LKS_CUDA(cudaMemcpy(b.p, p, N * 8, cudaMemcpyHostToDevice));
        LKS_CUDA(cudaMemcpy(b.p + N, u, (size_t)c->D * N * 8, cudaMemcpyHostToDevice));
        c->eng->import_state(c->g, b.p, b.p + N, c->d_init, 1.0 / 3.0, 0);
        LKS_CUDA(cudaDeviceSynchronize());
        c->custom_init = true;
    });
}

int lks_set_adjoint_terminal(lks_ctx* c, const double* lp, const double* lu) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if ((lp == nullptr) != (lu == nullptr)) throw LksError{LKS_EINVAL, "lam_p and lam_u must both be given or both NULL"};
        if (c->alks && lp) throw LksError{LKS_EINVAL, "the ALKS reverse sweep takes no terminal adjoint state"};
        drop_graphs(c);  // the captured reverse sweep starts from the previous terminal state
        c->have_forward = false;
        if (!lp) {
            c->custom_lterm = false;
            return;
        }
        const long long N = c->g.N;
        if (!c->d_lterm) c->d_lterm = dalloc(c, c->state_bytes);
        DevScratch b;
        LKS_CUDA(cudaMalloc(&b.p, (size_t)(c->D + 1) * N * 8));
        LKS_CUDA(cudaMemcpy(b.p, lp, N * 8, cudaMemcpyHostToDevice));
        LKS_CUDA(cudaMemcpy(b.p + N, lu, (size_t)c->D * N * 8, cudaMemcpyHostToDevice));
        c->eng->import_state(c->g, b.p, b.p + N, c->d_lterm, 0.0, 0);
        LKS_CUDA(cudaDeviceSynchronize());
        c->custom_lterm = true;
    });
}

int lks_get_adjoint_initial(lks_ctx* c, double* lp, double* lu) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!lp || !lu) throw LksError{LKS_EINVAL, "null pointer"};
        if (!c->have_lambda0) throw LksError{LKS_ESTATE, "no adjoint has run"};
        const long long N = c->g.N;
        DevScratch b;
        LKS_CUDA(cudaMalloc(&b.p, (size_t)(c->D + 1) * N * 8));
        LKS_CUDA(cudaDeviceSynchronize());
        c->eng->export_state(c->g, c->lam[0], b.p, b.p + N, 0.0, 0);
        LKS_CUDA(cudaMemcpy(lp, b.p, N * 8, cudaMemcpyDeviceToHost));
        LKS_CUDA(cudaMemcpy(lu, b.p + N, (size_t)c->D * N * 8, cudaMemcpyDeviceToHost));
    });
}

int lks_set_angle_knots(lks_ctx* c, const double* aknots) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->rot) throw LksError{LKS_EINVAL, "the context has no rotating body (K_w = 0)"};
        if (!aknots) throw LksError{LKS_EINVAL, "null pointer"};
        LKS_CUDA(cudaMemcpy(c->d_aknots, aknots, (size_t)c->prm.K_w * 8, cudaMemcpyHostToDevice));
    });
}

int lks_get_angle_gradient(lks_ctx* c, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->rot) throw LksError{LKS_EINVAL, "the context has no rotating body (K_w = 0)"};
        if (!out) throw LksError{LKS_EINVAL, "null pointer"};
        if (!c->have_lambda0) throw LksError{LKS_ESTATE, "no adjoint has run"};
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(out, c->d_out_a, (size_t)c->prm.K_w * 8, cudaMemcpyDeviceToHost));
    });
}

int lks_get_angles(lks_ctx* c, double* th, double* om) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->rot) throw LksError{LKS_EINVAL, "the context has no rotating body (K_w = 0)"};
        if (!th || !om) throw LksError{LKS_EINVAL, "null pointer"};
        if (!c->have_final) throw LksError{LKS_ESTATE, "no forward has run"};
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(th, c->d_theta, (size_t)(c->prm.Nt + 1) * 8, cudaMemcpyDeviceToHost));
        LKS_CUDA(cudaMemcpy(om, c->d_omega, (size_t)(c->prm.Nt + 1) * 8, cudaMemcpyDeviceToHost));
    });
}

int lks_angles_T(lks_ctx* c, const double* gth, const double* gom, double* out) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->rot) throw LksError{LKS_EINVAL, "the context has no rotating body (K_w = 0)"};
        if (!gth || !gom || !out) throw LksError{LKS_EINVAL, "null pointer"};
        const int Nt = c->prm.Nt, Kw = c->prm.K_w;
        DevScratch b;
        LKS_CUDA(cudaMalloc(&b.p, (size_t)(2 * (Nt + 1) + 2 * Kw) * 8));
        double *dth = b.p, *dom = b.p + (Nt + 1), *dt = b.p + 2 * (Nt + 1), *dout = dt + Kw;
        LKS_CUDA(cudaMemcpy(dth, gth, (size_t)(Nt + 1) * 8, cudaMemcpyHostToDevice));
        LKS_CUDA(cudaMemcpy(dom, gom, (size_t)(Nt + 1) * 8, cudaMemcpyHostToDevice));
        interp_T_kernel<<<nblk(Kw, 64), 64>>>(c->mgw, dth, dom, dt);
        LKS_LAUNCHED();
        motion_filter_kernel<<<nblk(Kw, 64), 64>>>(c->mgw, dt, c->d_anorm, dout, 1);
        LKS_LAUNCHED();
        LKS_CUDA(cudaMemcpy(out, dout, (size_t)Kw * 8, cudaMemcpyDeviceToHost));
    });
}

int lks_get_step_angle_sensitivities(lks_ctx* c, double* gth, double* gom) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->rot) throw LksError{LKS_EINVAL, "the context has no rotating body (K_w = 0)"};
        if (!gth || !gom) throw LksError{LKS_EINVAL, "null pointer"};
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(gth, c->d_gth, (size_t)(c->prm.Nt + 1) * 8, cudaMemcpyDeviceToHost));
        LKS_CUDA(cudaMemcpy(gom, c->d_gom, (size_t)(c->prm.Nt + 1) * 8, cudaMemcpyDeviceToHost));
    });
}

int lks_set_graphs(lks_ctx* c, int enable) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        drop_graphs(c);
        c->use_graphs = enable != 0;
        c->have_forward = false;
    });
}

int lks_get_status(lks_ctx* c) {
    if (!c) return LKS_EINVAL;
    return guard(c, [&] {
        if (!c->have_final) throw LksError{LKS_ESTATE, "no forward has run"};
        LKS_CUDA(cudaEventSynchronize(c->ev_flag));
        // the status word covers every kernel queued so far on any stream
        LKS_CUDA(cudaDeviceSynchronize());
        LKS_CUDA(cudaMemcpy(c->h_flag + 1, c->d_flag + 1, 4, cudaMemcpyDeviceToHost));
        check_flags(c);
    });
}

int lks_get_stats(const lks_ctx* c, lks_stats* out) {
    if (!c || !out) return LKS_EINVAL;
    *out = c->stats;
    return LKS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Density filter without any allocation.  Its only scratch (the per-node sum of filter weights) lives in
// a fixed file-scope device array; every GPU that loads the library holds that array until the process
// exits.  Host code must not pass the array's name to a kernel: on the host it names a stand-in object,
// so the device address is looked up once per device with cudaGetSymbolAddress.
// ------------------------------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_filter_norm[LKS_NOALLOC_FILTER_MAX];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_noalloc_err;
}  // namespace

extern "C" int lks_density_filter_noalloc(const int32_t nd[3], double R, const double* d_in, double* d_out,
                                          void* stream) {
    if (!nd || !d_in || !d_out) {
        g_noalloc_err = "null pointer";
        return LKS_EINVAL;
    }
    // the product is checked after every factor: it stays below 2^20 * 2^31 before the check, so it cannot overflow
    long long n = 1;
    for (int a = 0; a < 3; ++a) {
        if (nd[a] < 1) {
            g_noalloc_err = "design extents must be >= 1";
            return LKS_EINVAL;
        }
        n *= nd[a];
        if (n > LKS_NOALLOC_FILTER_MAX) {
            g_noalloc_err = "design grid of " + std::to_string(nd[0]) + " x " + std::to_string(nd[1]) + " x " +
                            std::to_string(nd[2]) + " nodes exceeds LKS_NOALLOC_FILTER_MAX (" +
                            std::to_string((long long)LKS_NOALLOC_FILTER_MAX) + ")";
            return LKS_EINVAL;
        }
    }
    if (!(R >= 0.0) || R > 32.0) {
        g_noalloc_err = "filter radius out of range [0, 32]";
        return LKS_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        g_noalloc_err = "no usable current CUDA device";
        return LKS_ECUDA;
    }
    double* norm = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // one-time set-up on this device (the device is current): the device address of the scratch array
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_filter_norm);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                g_noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LKS_ECUDA;
            }
            g_noalloc_ptr[dev] = (double*)p;
        }
        norm = g_noalloc_ptr[dev];
    }
    DesignGeom dg;
    std::memset(&dg, 0, sizeof(dg));
    for (int a = 0; a < 3; ++a) {
        dg.nd[a] = nd[a];
        dg.nde[a] = nd[a];
    }
    dg.R = R;
    cudaStream_t s = (cudaStream_t)stream;
    // the norm kernel overwrites every entry the filter reads, so nothing needs clearing between calls
    filter_norm_kernel<<<nblk(n, 128), 128, cone_table_bytes(R), s>>>(dg, norm);
    density_filter_kernel<<<nblk(n, 128), 128, cone_table_bytes(R), s>>>(dg, d_in, norm, d_out, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("kernel launch: ") + cudaGetErrorString(e);
        return LKS_ECUDA;
    }
    return LKS_OK;
}

extern "C" const char* lks_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

// ------------------------------------------------------------------------------------------------
// Batched parameter study: one graph for the forward sweeps of all instances, one for their reverse sweeps.
// ------------------------------------------------------------------------------------------------
struct lks_batch {
    std::vector<lks_ctx*> ctx;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gx_fwd = nullptr, gx_adj = nullptr;
    std::string err;
};

namespace {

template <typename F>
void batch_graph(lks_batch* b, cudaGraphExec_t& gx, cudaStream_t s, F&& body) {
    if (!gx) {
        LKS_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        try {
            LKS_CUDA(cudaEventRecord(b->ev, b->cap));
            for (lks_ctx* c : b->ctx) LKS_CUDA(cudaStreamWaitEvent(c->cap, b->ev, 0));
            for (lks_ctx* c : b->ctx) {
                body(c, c->cap);
                LKS_CUDA(cudaEventRecord(b->ev, c->cap));
                LKS_CUDA(cudaStreamWaitEvent(b->cap, b->ev, 0));
            }
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(b->cap, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        cudaGraph_t g = nullptr;
        LKS_CUDA(cudaStreamEndCapture(b->cap, &g));
        cudaError_t e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        LKS_CUDA(e);
    }
    LKS_CUDA(cudaGraphLaunch(gx, s));
}

void batch_free(lks_batch* b) {
    if (b->gx_fwd) cudaGraphExecDestroy(b->gx_fwd);
    if (b->gx_adj) cudaGraphExecDestroy(b->gx_adj);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (lks_ctx* c : b->ctx) lks_destroy(c);
    b->ctx.clear();
}

template <typename F>
int batch_guard(lks_batch* b, F&& f) {
    try {
        f();
        return LKS_OK;
    } catch (const LksError& e) {
        b->err = e.msg;
        return e.code;
    } catch (...) {
        b->err = "unexpected exception";
        return LKS_ECUDA;
    }
}

}  // namespace

extern "C" {

int lks_batch_create(int count, const lks_params* params, lks_batch** out) {
    if (count < 1 || !params || !out) return LKS_EINVAL;
    lks_batch* b = new lks_batch();
    int rc = LKS_OK;
    for (int i = 0; i < count && rc == LKS_OK; ++i) {
        if (params[i].Nt != params[0].Nt) {
            g_create_err = "all instances of a batch need the same Nt";
            rc = LKS_EINVAL;
            break;
        }
        lks_ctx* c = nullptr;
        rc = create_ctx(&params[i], true, &c);
        if (rc == LKS_OK) {
            c->use_graphs = false;  // the batch owns the graphs
            b->ctx.push_back(c);
        } else {
            g_create_err = "instance " + std::to_string(i) + ": " + g_create_err;
        }
    }
    if (rc == LKS_OK) {
        if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
            g_create_err = "stream/event creation failed";
            rc = LKS_ECUDA;
        }
    }
    if (rc != LKS_OK) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return LKS_OK;
}

void lks_batch_destroy(lks_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

lks_ctx* lks_batch_context(lks_batch* b, int index) {
    if (!b || index < 0 || index >= (int)b->ctx.size()) return nullptr;
    return b->ctx[index];
}

const char* lks_batch_last_error(const lks_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int lks_batch_forward_dev(lks_batch* b, const double* const* d_gamma, const double* const* d_pos, double* d_J,
                          void* stream) {
    if (!b || !d_gamma || !d_pos) return LKS_EINVAL;
    return batch_guard(b, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            lks_ctx* c = b->ctx[i];
            if (!d_gamma[i] || !d_pos[i]) throw LksError{LKS_EINVAL, "null input pointer of instance " + std::to_string(i)};
            LKS_CUDA(cudaMemcpyAsync(c->d_gamma, d_gamma[i], c->nd * 8, cudaMemcpyDeviceToDevice, s));
            LKS_CUDA(cudaMemcpyAsync(c->d_knots, d_pos[i], (size_t)c->prm.K * c->D * 8, cudaMemcpyDeviceToDevice, s));
        }
        batch_graph(b, b->gx_fwd, s, [&](lks_ctx* c, cudaStream_t cs) { forward_body(c, cs); });
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            lks_ctx* c = b->ctx[i];
            LKS_CUDA(cudaEventRecord(c->ev_flag, s));
            c->stats.forward_steps = c->prm.Nt;
            c->have_forward = true;
            if (d_J) LKS_CUDA(cudaMemcpyAsync(d_J + i, c->d_J, 8, cudaMemcpyDeviceToDevice, s));
        }
    });
}

int lks_batch_adjoint_dev(lks_batch* b, double* const* d_dgamma, double* const* d_dpos, void* stream) {
    if (!b) return LKS_EINVAL;
    return batch_guard(b, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            lks_ctx* c = b->ctx[i];
            if (!c->have_forward) throw LksError{LKS_ESTATE, "lks_batch_adjoint needs a preceding lks_batch_forward"};
        }
        batch_graph(b, b->gx_adj, s, [&](lks_ctx* c, cudaStream_t cs) { adjoint_body(c, cs); });
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            lks_ctx* c = b->ctx[i];
            finish_adjoint(c, d_dgamma ? d_dgamma[i] : nullptr, d_dpos ? d_dpos[i] : nullptr, s);
            poison_if_unstable(c, d_dgamma ? d_dgamma[i] : nullptr, d_dpos ? d_dpos[i] : nullptr, s);
            c->have_lambda0 = true;
            if (c->prm.ckpt == LKS_CKPT_REVOLVE) c->have_forward = false;
        }
    });
}

}  // extern "C"
