// D2Q9 engine (see lks_engine.cuh).
#pragma once

#include "lks_engine.cuh"
#include "lks_step2d.cuh"
#include "lks_step2r.cuh"
#include "lks_step2v.cuh"

namespace lks {

// D2Q9 engine with four kernel families: rows = 1 or 2 select the row-tile kernels (blocks of 32 x 8 threads,
// tiles 28 wide and 8 or 16 rows high; best on small grids, where launches are latency bound), rows = 3 the
// forward kernel that takes two steps per launch on 24 x 8 row tiles, rows = 4, 8, 16 the warp-column kernels
// with that many rows per warp and WY = 4 warps per block, rows = 32, 64 the vectorised warp columns (two grid
// columns per lane, 60 columns per warp).
template <typename T, int HW>
struct Engine2D : EngineCommon<T, 2, HW> {
    static constexpr int WY = 4;
    explicit Engine2D(const Geom& g) {
        LKS_CUDA(cudaFuncSetAttribute(fwd2r2_kernel<T, HW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r2_fwd<T>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd2r2_kernel<T, HW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r2_fwd<T>()));
        LKS_CUDA(cudaFuncSetAttribute(adj2r2_kernel<T, HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r2_adj<T>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd2r_kernel<T, HW, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r_fwd<T, 1>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd2r_kernel<T, HW, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r_fwd<T, 2>()));
        LKS_CUDA(cudaFuncSetAttribute(adj2r_kernel<T, HW, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r_adj<T, 1>()));
        LKS_CUDA(cudaFuncSetAttribute(adj2r_kernel<T, HW, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2r_adj<T, 2>()));
        LKS_CUDA(cudaFuncSetAttribute(adj2v_kernel<T, HW, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Adj2vRing<T>::bytes()));
        LKS_CUDA(cudaFuncSetAttribute(adj2v_kernel<T, HW, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Adj2vRing<T>::bytes()));
        this->alks_attr();
        set_rows(1, 1, g);
    }
    static void geom(int r, const Geom& g, dim3& th, dim3& tile, dim3& grid) {
        if (r >= 32) {  // vectorised warp columns, two columns per lane
            th = dim3(32 * WY, 1, 1);
            tile = dim3(kVecCols, r * WY, 1);
            grid = dim3(nblk(g.n[0], kVecCols), nblk(g.n[1], r * WY), 1);
        } else if (r == 3) {  // two-step fused row tiles
            th = dim3(32, 8, 1);
            tile = dim3(Fused2::TXO, Fused2::TY, 1);
            grid = dim3(nblk(g.n[0], Fused2::TXO), nblk(g.n[1], Fused2::TY), 1);
        } else if (r <= 2) {
            th = dim3(32, 8, 1);
            tile = dim3(28, 8 * r, 1);
            grid = dim3(nblk(g.n[0], 28), nblk(g.n[1], 8 * r), 1);
        } else {
            th = dim3(32 * WY, 1, 1);
            tile = dim3(kLanesOut, r * WY, 1);
            grid = dim3(nblk(g.n[0], kLanesOut), nblk(g.n[1], r * WY), 1);
        }
    }
    std::vector<int> fwd_codes() const override { return {1, 2, 3, 4, 8, 16, 32, 64}; }
    std::vector<int> adj_codes() const override { return {1, 2, 3, 4, 8, 16, 32, 64}; }
    bool set_rows(int rf, int ra, const Geom& g) override {
        // rows kept in registers grow with R: FP32 allows up to 16, FP64 up to 8 without spills; 3 = fused forward;
        // 32 and 64 = vectorised warp columns (even x extent only)
        // (the vectorised adjoint indexes in 32 bits: 3 N must fit)
        const bool even = (g.n[0] % 2) == 0, small = 3 * g.N < (1LL << 31);
        auto ok = [even, small](int r) {
            return r == 1 || r == 2 || r == 4 || r == 8 || (r == 16 && sizeof(T) == 4) ||
                   ((r == 32 || r == 64) && even && small);
        };
        if (!(ok(rf) || rf == 3) || !(ok(ra) || ra == 3)) return false;
        this->rows_f = rf;
        this->rows_a = ra;
        geom(rf, g, this->fthreads, this->ftile, this->fgrid);
        geom(ra, g, this->athreads, this->atile, this->agrid);
        return true;
    }
    template <int R>
    void fwd_r(const Geom& g, FwdArgs<T> a, cudaStream_t s) {
        launch_pdl(fwd2d_kernel<T, HW, R, WY>, this->fgrid, this->fthreads, 0, s, this->pdl, g, a);
    }
    bool fused2() const override { return this->rows_f == 3; }
    // FP32 state, hat kernel: the vectorised forward writes the footprint factors for the adjoint (map_hat2, the
    // arithmetic of box_fac below); the sensitivities and the design gather run as column kernels
    static constexpr bool kHat = kHat2f<T, HW>;
    bool fwd_writes_fac() const override { return kHat && (this->rows_f == 32 || this->rows_f == 64); }
    void box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                 cudaStream_t s) override {
        if constexpr (kHat) {
            box_fac_hat2_kernel<<<dim3(nblk(g.Fbn, 256), nsteps, 1), 256, 0, s>>>(g, poses, (const float*)kref, n_first,
                                                                                 (float*)out);
            LKS_LAUNCHED();
        } else {
            EngineCommon<T, 2, HW>::box_fac(g, poses, kref, n_first, nsteps, out, s);
        }
    }
    void sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride, int n_first,
              int nsteps, void* kbar, double* mslot, bool alks, cudaStream_t s) override {
        if constexpr (kHat) {
            if (!alks) {
                adj_sens_hat2_kernel<<<dim3(sens_blocks(g, alks), nsteps, 1), kSensHat2NT, 0, s>>>(
                    g, poses, (const float*)kref, (const float*)boxbuf, bstride, n_first, (float*)kbar, mslot);
                LKS_LAUNCHED();
                return;
            }
        }
        EngineCommon<T, 2, HW>::sens(g, poses, kref, boxbuf, bstride, n_first, nsteps, kbar, mslot, alks, s);
    }
    int sens_blocks(const Geom& g, bool alks) const override {
        if (kHat && !alks) return (int)(nblk(g.Fb[0], kSensHat2NT) * nblk(g.Fb[1], kSensHat2YC));
        return EngineCommon<T, 2, HW>::sens_blocks(g, alks);
    }
    void gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps, long long kstride,
                double* dkref, cudaStream_t s) override {
        if constexpr (kHat) {
            const long long nd = (long long)g.nde[0] * g.nde[1];
            design_gather_hat2_kernel<<<nblk(nd, kGatherHat2NT), kGatherHat2NT, 0, s>>>(g, poses, (const float*)kbar,
                                                                                     n_first, nsteps, kstride, dkref);
            LKS_LAUNCHED();
        } else {
            EngineCommon<T, 2, HW>::gather(g, poses, kbar, n_first, nsteps, kstride, dkref, s);
        }
    }
    bool fused_adj2() const override { return this->rows_a == 3; }
    void adj2(const Geom& g, const void* lam_in, void* lam_out, const void* prev1, const void* cur1, const void* prev2,
              const void* kref, const Pose* pose, void* boxbuf1, const void* fac1, int src1, void* boxbuf2,
              const void* fac2, int src2, cudaStream_t s) override;
    void fwd2(const Geom& g, const void* in, void* out1, void* out2, const void* kref, const Pose* pose1,
              double* jslot1, double* jslot2, unsigned* flag, const int* jlo, const int* jn, cudaStream_t s) override {
        auto a1 = make_fwd_args<T>(g, in, out1, kref, pose1, jslot1, flag, jlo, jn);
        auto a2 = make_fwd_args<T>(g, out1, out2 ? out2 : out1, kref, pose1 + 1, jslot2, flag, jlo, jn);
        fwd2r2(g, a1, a2, out2 ? 1 : 0, s);
    }
    // the squares of n.u are summed only when the objective has the variance term (a separate instantiation, so
    // that the plain objective keeps the kernel's code unchanged)
    void fwd2r2(const Geom& g, const FwdArgs<T>& a1, const FwdArgs<T>& a2, int two, cudaStream_t s) {
        if (a1.jsq != nullptr)
            launch_pdl(fwd2r2_kernel<T, HW, true>, this->fgrid, this->fthreads, smem2r2_fwd<T>(), s, this->pdl, g, a1,
                       a2, two);
        else
            launch_pdl(fwd2r2_kernel<T, HW, false>, this->fgrid, this->fthreads, smem2r2_fwd<T>(), s, this->pdl, g, a1,
                       a2, two);
    }
    template <int R>
    void adj_r(const Geom& g, AdjArgs<T> a, cudaStream_t s) {
        launch_pdl(adj2d_kernel<T, HW, R, WY>, this->agrid, this->athreads, 0, s, this->pdl, g, a);
    }
    void fwd(const Geom& g, const void* in, void* out, const void* kref, const Pose* pose, double* jslot,
             unsigned* flag, const int* jlo, const int* jn, cudaStream_t s) override {
        auto a = make_fwd_args<T>(g, in, out, kref, pose, jslot, flag, jlo, jn);
        if (this->rows_f == 32 || this->rows_f == 64) a.fac_out = (T*)this->fac_out;  // read by fwd2v (FP32, hat)
        switch (this->rows_f) {
            case 3:
                fwd2r2(g, a, a, 0, s);
                break;
            case 1: launch_pdl(fwd2r_kernel<T, HW, 1>, this->fgrid, this->fthreads, smem2r_fwd<T, 1>(), s, this->pdl, g, a); break;
            case 2: launch_pdl(fwd2r_kernel<T, HW, 2>, this->fgrid, this->fthreads, smem2r_fwd<T, 2>(), s, this->pdl, g, a); break;
            case 4: fwd_r<4>(g, a, s); break;
            case 8: fwd_r<8>(g, a, s); break;
            case 32: launch_pdl(fwd2v_kernel<T, HW, 32>, this->fgrid, this->fthreads, smem2v_fwd<T>(), s, this->pdl, g, a); break;
            case 64: launch_pdl(fwd2v_kernel<T, HW, 64>, this->fgrid, this->fthreads, smem2v_fwd<T>(), s, this->pdl, g, a); break;
            default: fwd_r<(sizeof(T) == 4 ? 16 : 8)>(g, a, s); break;
        }
    }
    void adj(const Geom& g, const void* lam_in, void* lam_out, const void* prev, const void* cur, const void* kref,
             const Pose* pose, void* boxbuf, const void* fac, int src, cudaStream_t s) override {
        auto a = make_adj_args<T>(g, lam_in, lam_out, prev, cur, kref, pose, boxbuf, fac, src);
        switch (this->rows_a) {
            case 3:
                launch_pdl(adj2r2_kernel<T, HW>, this->agrid, this->athreads, smem2r2_adj<T>(), s, this->pdl, g, a, a, 0);
                break;
            case 1: launch_pdl(adj2r_kernel<T, HW, 1>, this->agrid, this->athreads, smem2r_adj<T, 1>(), s, this->pdl, g, a); break;
            case 2: launch_pdl(adj2r_kernel<T, HW, 2>, this->agrid, this->athreads, smem2r_adj<T, 2>(), s, this->pdl, g, a); break;
            case 4: adj_r<4>(g, a, s); break;
            case 8: adj_r<8>(g, a, s); break;
            case 32: launch_pdl(adj2v_kernel<T, HW, 32>, this->agrid, this->athreads, Adj2vRing<T>::bytes(), s, this->pdl, g, a); break;
            case 64: launch_pdl(adj2v_kernel<T, HW, 64>, this->agrid, this->athreads, Adj2vRing<T>::bytes(), s, this->pdl, g, a); break;
            default: adj_r<(sizeof(T) == 4 ? 16 : 8)>(g, a, s); break;
        }
    }
};

template <typename T, int HW>
void Engine2D<T, HW>::adj2(const Geom& g, const void* lam_in, void* lam_out, const void* prev1, const void* cur1,
                           const void* prev2, const void* kref, const Pose* pose, void* boxbuf1, const void* fac1,
                           int src1, void* boxbuf2, const void* fac2, int src2, cudaStream_t s) {
    auto a1 = make_adj_args<T>(g, lam_in, lam_out, prev1, cur1, kref, pose, boxbuf1, fac1, src1);
    auto a2 = make_adj_args<T>(g, lam_in, lam_out, prev2, prev1, kref, pose - 1, boxbuf2, fac2, src2);
    launch_pdl(adj2r2_kernel<T, HW>, this->agrid, this->athreads, smem2r2_adj<T>(), s, this->pdl, g, a1, a2, 1);
}

}  // namespace lks
