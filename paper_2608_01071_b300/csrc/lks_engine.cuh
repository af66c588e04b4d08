// Step-kernel engines: the launches of the templated step, sensitivity and footprint kernels for one (precision,
// dimension, transfer-kernel width), behind a virtual interface that the host runtime (lks_api.cu) drives.  Each
// (lattice, precision) pair is compiled in a translation unit of its own (lks_engine_*.cu), in parallel.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lks.h"
#include "lks_common.cuh"
#include "lks_prep_kernels.cuh"
#include "lks_step_kernels.cuh"
#include "lks_oar.cuh"
#include "lks_rot.cuh"
#include "lks_oar_rot.cuh"
#include "lks_alks.cuh"

namespace lks {

struct LksError {
    int code;
    std::string msg;
};

#define LKS_CUDA(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            throw LksError{LKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};              \
    } while (0)

#define LKS_LAUNCHED()                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                                             \
        if (e_ != cudaSuccess) throw LksError{LKS_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)}; \
    } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Launch a step kernel with programmatic stream serialization (see pdl_wait_then_release).
template <typename K, typename... Args>
void launch_pdl(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess) throw LksError{LKS_ECUDA, std::string("cudaLaunchKernelEx: ") + cudaGetErrorString(e)};
}

// ------------------------------------------------------------------------------------------------
// Typed engine: launches of the templated kernels for one (precision, dimension, kernel width).
// ------------------------------------------------------------------------------------------------
struct Engine {
    bool pdl = true;  // programmatic dependent launch of the step kernels
    dim3 fthreads, athreads;  // threads per block of the forward / adjoint step kernels
    dim3 ftile, atile;        // analysis nodes covered per block
    dim3 fgrid, agrid;
    int rows_f = 0, rows_a = 0;  // step-kernel variant codes (tile_rows) of the forward / adjoint kernels
    virtual ~Engine() {}
    // choose the forward and adjoint step-kernel variants; false when one is not available for this grid
    virtual bool set_rows(int rf, int ra, const Geom& g) = 0;
    // variant codes the autotuner tries (some may be unavailable for a given grid)
    virtual std::vector<int> fwd_codes() const = 0;
    virtual std::vector<int> adj_codes() const = 0;
    virtual void fwd(const Geom& g, const void* in, void* out, const void* kref, const Pose* pose, double* jslot,
                     unsigned* flag, const int* jlo, const int* jn, cudaStream_t s) = 0;
    // two-step forward launches (steps n and n+1 in one kernel); out2 == nullptr takes step n only
    // 1 / (1 + kappa) of the step on the footprint box, written by the forward kernel for the adjoint when it can
    // (fwd_writes_fac) and this is set (for one fwd call)
    void* fac_out = nullptr;
    virtual bool fwd_writes_fac() const { return false; }
    virtual bool fused2() const { return false; }
    virtual void fwd2(const Geom& g, const void* in, void* out1, void* out2, const void* kref, const Pose* pose1,
                      double* jslot1, double* jslot2, unsigned* flag, const int* jlo, const int* jn, cudaStream_t s) {}
    // fac: 1 / (1 + kappa) of the step on the footprint box (box_fac), or nullptr to evaluate the mapping
    virtual void adj(const Geom& g, const void* lam_in, void* lam_out, const void* prev, const void* cur,
                     const void* kref, const Pose* pose, void* boxbuf, const void* fac, int src, cudaStream_t s) = 0;
    // two-step adjoint launches: steps n (pose, boxbuf1, src1; states prev1 = n-1, cur1 = n) and n-1 (pose - 1,
    // boxbuf2, src2; states prev2 = n-2, prev1) in one kernel
    virtual bool fused_adj2() const { return false; }
    virtual void adj2(const Geom& g, const void* lam_in, void* lam_out, const void* prev1, const void* cur1,
                      const void* prev2, const void* kref, const Pose* pose, void* boxbuf1, const void* fac1, int src1,
                      void* boxbuf2, const void* fac2, int src2, cudaStream_t s) {}
    // 1 / (1 + kappa) on the footprint box for steps n_first .. n_first + nsteps - 1 (stride Fbn per step)
    virtual void box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                         cudaStream_t s) = 0;
    virtual void sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride,
                      int n_first, int nsteps, void* kbar, double* mslot, bool alks, cudaStream_t s) = 0;
    // blocks per step of sens (the motion partials per step in mslot)
    virtual int sens_blocks(const Geom& g, bool alks) const { return (int)nblk(g.Fbn, 256 * kSensNPT); }
    // the ALKS reverse sweep (lks_alks.cuh): terminal state and one step; the pointers of AlksArgs are in the state
    // precision of the engine
    virtual void alks_init(const Geom& g, const Pose* pose, const void* kref, void* lam, const void* args,
                           cudaStream_t s) = 0;
    virtual void alks_step(const Geom& g, const void* args, cudaStream_t s) = 0;
    virtual void gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps,
                        long long kstride, double* dkref, cudaStream_t s) = 0;
    virtual void kappa_ref(const DesignGeom& dg, const double* gt, double* gb, double* k64, void* k, cudaStream_t s) = 0;
    virtual void init_state(const Geom& g, void* st, cudaStream_t s) = 0;
    virtual void import_state(const Geom& g, const double* p, const double* u, void* st, double pshift,
                              cudaStream_t s) = 0;
    virtual void add_state(const Geom& g, void* dst, const void* src, cudaStream_t s) = 0;
    virtual void init_adjoint(const Geom& g, const void* fin, void* lam, int src, cudaStream_t s) = 0;
    // objective J2 (translating body): per-block partials of sum_x kappa u of one step, and its adjoint source
    virtual void oar_partial(const Geom& g, const Pose* pose, const void* kref, const void* st, double* scratch,
                             unsigned* ticket, double* slot, cudaStream_t s) = 0;
    virtual void oar_source(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, void* lam,
                            cudaStream_t s) = 0;
    virtual void oar_sens(const Geom& g, const OarGeom& o, const Pose* poses, const void* kref, const void* boxbuf,
                          long long bstride, int n_first, int nsteps, void* kbar, double* scratch, unsigned* tickets,
                          double* oms, cudaStream_t s) = 0;
    // objective J2 with a rotating body (lks_oar_rot.cuh): the per-step design-side sums and the compensated
    // d j2 / d kappa^ref accumulation (kh, kl: state precision, extended design grid); the adjoint source
    virtual void oar_rot_partial(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, const void* st,
                                 void* kh, void* kl, double* scratch, unsigned* ticket, double* slot, cudaStream_t s) = 0;
    virtual void oar_rot_source(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, void* lam,
                                cudaStream_t s) = 0;
    virtual void export_state(const Geom& g, const void* st, double* p, double* u, double pshift, cudaStream_t s) = 0;
    // rotating body (lks_rot.cuh): kappa and u^S of one step on the footprint box; 1 / (1 + kappa) for a segment's
    // steps; the local sensitivities of a segment (kappa-bar, u^S-bar per box node, per-block motion partials); the
    // transposed mapping on the design side; the per-step motion sums
    virtual void rot_box_map(const Geom& g, const Pose* pose, const void* kref, void* map, cudaStream_t s) = 0;
    virtual void rot_box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                             cudaStream_t s) = 0;
    virtual void rot_sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride,
                          int n_first, int nsteps, void* kbar, double* mslot, cudaStream_t s) = 0;
    virtual void rot_gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps,
                            long long kstride, double* dkref, cudaStream_t s) = 0;
};

template <typename T>
FwdArgs<T> make_fwd_args(const Geom& g, const void* in, void* out, const void* kref, const Pose* pose, double* jslot,
                         unsigned* flag, const int* jlo, const int* jn) {
    FwdArgs<T> a;
    for (int i = 0; i < 3; ++i) {
        a.jb_lo[i] = jlo[i];
        a.jb_n[i] = jn[i];
        a.dir[i] = (T)g.dir[i];
    }
    a.in = (const T*)in;
    a.out_p = (T*)out;
    a.out_u = (T*)out + g.N;
    a.kref = (const T*)kref;
    a.pose = pose;
    a.jslot = jslot;
    a.jsq = jslot != nullptr && g.jsq_off != 0 ? jslot + g.jsq_off : nullptr;
    a.flag = flag;
    a.fac_out = nullptr;
    a.u_crit2 = (T)g.u_crit2;
    return a;
}

template <typename T>
AdjArgs<T> make_adj_args(const Geom& g, const void* lam_in, void* lam_out, const void* prev, const void* cur,
                         const void* kref, const Pose* pose, void* boxbuf, const void* fac, int src) {
    AdjArgs<T> a;
    a.lam_in = (const T*)lam_in;
    a.lam_out = (T*)lam_out;
    a.u_prev = (const T*)prev + g.N;
    a.u_cur = (const T*)cur + g.N;
    a.kref = (const T*)kref;
    a.pose = pose;
    a.boxbuf = (T*)boxbuf;
    a.fac = (const T*)fac;
    a.src = src;
    for (int i = 0; i < 3; ++i) {
        a.phi_dir[i] = (T)(g.dir[i] * g.phi);
        a.dir[i] = (T)g.dir[i];
    }
    a.src_c0 = g.phi_var != 0.0 ? g.obj + 3 : nullptr;
    a.src_c1 = (T)(2.0 * g.phi_var);
    return a;
}

// Shared pieces of both engines.
template <typename T, int D, int HW>
struct EngineCommon : Engine {
    void box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                 cudaStream_t s) override {
        box_fac_kernel<T, D, HW><<<dim3(nblk(g.Fbn, 256), nsteps, 1), 256, 0, s>>>(g, poses, (const T*)kref, n_first,
                                                                                 (T*)out);
        LKS_LAUNCHED();
    }
    void sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride, int n_first,
              int nsteps, void* kbar, double* mslot, bool alks, cudaStream_t s) override {
        const dim3 grid(nblk(g.Fbn, 256 * kSensNPT), nsteps, 1);
        if (alks)
            adj_sens_kernel<T, D, HW, true><<<grid, 256, 0, s>>>(g, poses, (const T*)kref, (const T*)boxbuf, bstride,
                                                                 n_first, (T*)kbar, mslot);
        else
            adj_sens_kernel<T, D, HW><<<grid, 256, 0, s>>>(g, poses, (const T*)kref, (const T*)boxbuf, bstride, n_first,
                                                           (T*)kbar, mslot);
        LKS_LAUNCHED();
    }
    // ALKS tiles: 32 x 8 nodes in 2D, 32 x 4 x 4 in 3D
    static constexpr int ATX = 32, ATY = D == 2 ? 8 : 4, ATZ = D == 2 ? 1 : 4;
    static constexpr size_t alks_smem() {
        using TL = Tile<D, ATX, ATY, ATZ>;
        return sizeof(T) * (AlksState<D>::NS * TL::S + (1 + D) * TL::M);
    }
    void alks_init(const Geom& g, const Pose* pose, const void* kref, void* lam, const void* args,
                   cudaStream_t s) override {
        alks_init_kernel<T, D, HW><<<nblk(g.N, 256), 256, 0, s>>>(g, pose, (const T*)kref, (T*)lam,
                                                                  *(const AlksArgs<T>*)args);
        LKS_LAUNCHED();
    }
    // called by the engines' constructors (the tiles' shared memory exceeds the default limit)
    void alks_attr() {
        LKS_CUDA(cudaFuncSetAttribute(alks_step_kernel<T, D, HW, ATX, ATY, ATZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)alks_smem()));
    }
    void alks_step(const Geom& g, const void* args, cudaStream_t s) override {
        const dim3 grid(nblk(g.n[0], ATX), nblk(g.n[1], ATY), nblk(g.n[2], ATZ));
        launch_pdl(alks_step_kernel<T, D, HW, ATX, ATY, ATZ>, grid, dim3(ATX, ATY, ATZ), alks_smem(), s, this->pdl, g,
                   *(const AlksArgs<T>*)args);
    }
    void gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps, long long kstride,
                double* dkref, cudaStream_t s) override {
        const long long nd = (long long)g.nde[0] * g.nde[1] * g.nde[2];
        design_gather_kernel<T, D, HW><<<nblk(nd, 128), 128, 0, s>>>(g, poses, (const T*)kbar, n_first, nsteps, kstride, dkref);
        LKS_LAUNCHED();
    }
    void kappa_ref(const DesignGeom& dg, const double* gt, double* gb, double* k64, void* k, cudaStream_t s) override {
        const long long ne = (long long)dg.nde[0] * dg.nde[1] * dg.nde[2];
        kappa_ref_kernel<T><<<nblk(ne, 256), 256, 0, s>>>(dg, gt, gb, k64, (T*)k);
        LKS_LAUNCHED();
    }
    void init_state(const Geom& g, void* st, cudaStream_t s) override {
        init_state_kernel<T, D><<<nblk(g.N, 256), 256, 0, s>>>(g, (T*)st);
        LKS_LAUNCHED();
    }
    void import_state(const Geom& g, const double* p, const double* u, void* st, double pshift,
                      cudaStream_t s) override {
        import_state_kernel<T, D><<<nblk(g.N, 256), 256, 0, s>>>(g, p, u, (T*)st, pshift);
        LKS_LAUNCHED();
    }
    void add_state(const Geom& g, void* dst, const void* src, cudaStream_t s) override {
        add_state_kernel<T, D><<<nblk((D + 1) * g.N, 256), 256, 0, s>>>(g, (T*)dst, (const T*)src);
        LKS_LAUNCHED();
    }
    void init_adjoint(const Geom& g, const void* fin, void* lam, int src, cudaStream_t s) override {
        init_adjoint_kernel<T, D><<<nblk(g.N, 256), 256, 0, s>>>(g, (const T*)fin + g.N, (T*)lam, src);
        LKS_LAUNCHED();
    }
    void export_state(const Geom& g, const void* st, double* p, double* u, double pshift, cudaStream_t s) override {
        export_state_kernel<T, D><<<nblk(g.N, 256), 256, 0, s>>>(g, (const T*)st, p, u, pshift);
        LKS_LAUNCHED();
    }
    void rot_box_map(const Geom& g, const Pose* pose, const void* kref, void* map, cudaStream_t s) override {
        rot_box_map_kernel<T, D, HW><<<nblk(g.Fbn, 256), 256, 0, s>>>(g, pose, (const T*)kref, (T*)map);
        LKS_LAUNCHED();
    }
    void rot_box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                     cudaStream_t s) override {
        rot_box_fac_kernel<T, D, HW><<<dim3(nblk(g.Fbn, 256), nsteps, 1), 256, 0, s>>>(g, poses, (const T*)kref, n_first,
                                                                                     (T*)out);
        LKS_LAUNCHED();
    }
    void rot_sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride, int n_first,
                  int nsteps, void* kbar, double* mslot, cudaStream_t s) override {
        rot_sens_kernel<T, D, HW><<<dim3(nblk(g.Fbn, 256), nsteps, 1), 256, 0, s>>>(
            g, poses, (const T*)kref, (const T*)boxbuf, bstride, n_first, (T*)kbar, mslot);
        LKS_LAUNCHED();
    }
    void rot_gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps, long long kstride,
                    double* dkref, cudaStream_t s) override {
        const long long nd = (long long)g.nde[0] * g.nde[1] * g.nde[2];
        rot_gather_kernel<T, D, HW><<<nblk(nd, 128), 128, 0, s>>>(g, poses, (const T*)kbar, n_first, nsteps, kstride, dkref);
        LKS_LAUNCHED();
    }
    void oar_partial(const Geom& g, const Pose* pose, const void* kref, const void* st, double* scratch,
                     unsigned* ticket, double* slot, cudaStream_t s) override {
        oar_partial_kernel<T, D, HW><<<nblk(g.Fbn, 256), 256, 0, s>>>(g, pose, (const T*)kref, (const T*)st, scratch,
                                                                     ticket, slot);
        LKS_LAUNCHED();
    }
    void oar_rot_partial(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, const void* st, void* kh,
                         void* kl, double* scratch, unsigned* ticket, double* slot, cudaStream_t s) override {
        const long long nd = (long long)g.nde[0] * g.nde[1] * g.nde[2];
        oar_rot_partial_kernel<T, D, HW><<<nblk(nd, 256), 256, 0, s>>>(g, o, pose, (const T*)kref, (const T*)st, (T*)kh,
                                                                       (T*)kl, scratch, ticket, slot);
        LKS_LAUNCHED();
    }
    void oar_rot_source(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, void* lam,
                        cudaStream_t s) override {
        oar_rot_source_kernel<T, D, HW><<<nblk(g.Fbn, 256), 256, 0, s>>>(g, o, pose, (const T*)kref, (T*)lam);
        LKS_LAUNCHED();
    }
    void oar_source(const Geom& g, const OarGeom& o, const Pose* pose, const void* kref, void* lam,
                    cudaStream_t s) override {
        oar_source_kernel<T, D, HW><<<nblk(g.Fbn, 256), 256, 0, s>>>(g, o, pose, (const T*)kref, (T*)lam);
        LKS_LAUNCHED();
    }
    void oar_sens(const Geom& g, const OarGeom& o, const Pose* poses, const void* kref, const void* boxbuf,
                  long long bstride, int n_first, int nsteps, void* kbar, double* scratch, unsigned* tickets,
                  double* oms, cudaStream_t s) override {
        const dim3 grid(nblk(g.Fbn, 256), nsteps, 1);
        oar_sens_kernel<T, D, HW><<<grid, 256, 0, s>>>(g, o, poses, (const T*)kref, (const T*)boxbuf, bstride, n_first,
                                                       (T*)kbar, scratch, tickets, oms);
        LKS_LAUNCHED();
    }
};

// One engine per (lattice, precision); hw = 1 (hat) or 2 (cosine transfer kernel).  Internal to the library: hidden
// from its dynamic symbol table, which holds the C ABI alone.
#define LKS_INTERNAL __attribute__((visibility("hidden")))
LKS_INTERNAL Engine* make_engine2d_f32(int hw, const Geom& g);
LKS_INTERNAL Engine* make_engine2d_f64(int hw, const Geom& g);
LKS_INTERNAL Engine* make_engine3d_f32(int hw, const Geom& g);
LKS_INTERNAL Engine* make_engine3d_f64(int hw, const Geom& g);

}  // namespace lks
