// D3Q15 engine (see lks_engine.cuh).
#pragma once

#include "lks_engine.cuh"
#include "lks_step3d.cuh"
#include "lks_step3s.cuh"
#include "lks_step3p.cuh"

#include <type_traits>

namespace lks {

// D3Q15 engine: rows = 1 selects the generic shared-memory tile kernels (32 x 4 x 4 nodes per block);
// rows = 8 or 16 the z-marching kernels with that many planes per block (32 x 8 columns); forward rows = 32,
// 64 the separable z-marching kernels with 16 or 32 planes per block (32 x 8 columns), forward rows = 96 the
// separable forward with 16 planes of 32 x 16 columns; FP32 rows = 128, 160 the plane-pair separable kernels (packed
// FP32x2, forward and adjoint) with 16 or 32 planes per block (32 x 8 columns).
template <typename T, int HW>
struct Engine3D : EngineCommon<T, 3, HW> {
    static constexpr int TX = 32, TY = 4, TZ = 4;
    using TL = Tile<3, TX, TY, TZ>;
    static constexpr size_t smem_fwd = sizeof(T) * (4 * TL::S + 7 * TL::M);
    static constexpr size_t smem_adj = sizeof(T) * (4 * TL::S + 10 * TL::M);

    explicit Engine3D(const Geom& g) {
        LKS_CUDA(cudaFuncSetAttribute(fwd_step_kernel<T, 3, HW, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_fwd));
        LKS_CUDA(cudaFuncSetAttribute(adj_step_kernel<T, 3, HW, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_adj));
        LKS_CUDA(cudaFuncSetAttribute(fwd3d_kernel<T, HW, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3d_fwd<T>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd3d_kernel<T, HW, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3d_fwd<T>()));
        LKS_CUDA(cudaFuncSetAttribute(adj3d_kernel<T, HW, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3d_adj<T>()));
        LKS_CUDA(cudaFuncSetAttribute(adj3d_kernel<T, HW, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3d_adj<T>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd3s_kernel<T, HW, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem3s_fwd<T, 8>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd3s_kernel<T, HW, 32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem3s_fwd<T, 8>()));
        LKS_CUDA(cudaFuncSetAttribute(fwd3s_kernel<T, HW, 16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem3s_fwd<T, 16>()));
        LKS_CUDA(cudaFuncSetAttribute(adj3s_kernel<T, HW, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem3s_adj<T, 8>()));
        LKS_CUDA(cudaFuncSetAttribute(adj3s_kernel<T, HW, 32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem3s_adj<T, 8>()));
        if constexpr (kPair) {
            const int sm = (int)smem3p_fwd();
            LKS_CUDA(cudaFuncSetAttribute(fwd3p_kernel<HW, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            LKS_CUDA(cudaFuncSetAttribute(fwd3p_kernel<HW, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            LKS_CUDA(cudaFuncSetAttribute(fwd3p_kernel<HW, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            LKS_CUDA(cudaFuncSetAttribute(fwd3p_kernel<HW, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
            const int sa = (int)smem3p_adj();
            LKS_CUDA(cudaFuncSetAttribute(adj3p_kernel<HW, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
            LKS_CUDA(cudaFuncSetAttribute(adj3p_kernel<HW, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
            LKS_CUDA(cudaFuncSetAttribute(adj3p_kernel<HW, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
            LKS_CUDA(cudaFuncSetAttribute(adj3p_kernel<HW, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
        }
        this->alks_attr();
        set_rows(8, 8, g);
    }
    // the plane-pair kernels exist for the FP32 state only
    static constexpr bool kPair = std::is_same<T, float>::value;
    std::vector<int> fwd_codes() const override {
        if (kPair) return {1, 8, 16, 32, 64, 96, 128, 160};
        return {1, 8, 16, 32, 64, 96};
    }
    std::vector<int> adj_codes() const override {
        if (kPair) return {1, 8, 16, 32, 64, 128, 160};
        return {1, 8, 16, 32, 64};
    }
    static void geom(int r, const Geom& g, dim3& th, dim3& tile, dim3& grid) {
        if (r == 1) {
            th = tile = dim3(TX, TY, TZ);
            grid = dim3(nblk(g.n[0], TX), nblk(g.n[1], TY), nblk(g.n[2], TZ));
        } else if (r >= 128) {  // plane-pair separable forward: 16 or 32 planes of 32 x 8 columns
            const int zb = r == 160 ? 32 : 16;
            th = dim3(Pair3::TX, Pair3::TY, 1);
            tile = dim3(Pair3::TX, Pair3::TY, zb);
            grid = dim3(nblk(g.n[0], Pair3::TX), nblk(g.n[1], Pair3::TY), nblk(g.n[2], zb));
        } else if (r >= 32) {  // separable forward: (planes, rows) per block
            const int zb = r == 64 ? 32 : 16, ty = r == 96 ? 16 : 8;
            th = dim3(32, ty, 1);
            tile = dim3(32, ty, zb);
            grid = dim3(nblk(g.n[0], 32), nblk(g.n[1], ty), nblk(g.n[2], zb));
        } else {
            th = dim3(Reg3::TX, Reg3::TY, 1);
            tile = dim3(Reg3::TX, Reg3::TY, r);
            grid = dim3(nblk(g.n[0], Reg3::TX), nblk(g.n[1], Reg3::TY), nblk(g.n[2], r));
        }
    }
    bool set_rows(int rf, int ra, const Geom& g) override {
        auto okf = [](int r) { return r == 1 || r == 8 || r == 16 || r == 32 || r == 64 || r == 96 || (kPair && (r == 128 || r == 160)); };
        auto oka = [](int r) { return r == 1 || r == 8 || r == 16 || r == 32 || r == 64 || (kPair && (r == 128 || r == 160)); };
        if (!okf(rf) || !oka(ra)) return false;
        // the plane-pair kernels index in 32 bits: every field offset c N + i and box offset c Fbn + b must fit
        const bool small = 4 * g.N < (1LL << 31) && 6 * g.Fbn < (1LL << 31);
        if (!small && (rf >= 128 || ra >= 128)) return false;
        this->rows_f = rf;
        this->rows_a = ra;
        geom(rf, g, this->fthreads, this->ftile, this->fgrid);
        geom(ra, g, this->athreads, this->atile, this->agrid);
        return true;
    }
    void fwd(const Geom& g, const void* in, void* out, const void* kref, const Pose* pose, double* jslot,
             unsigned* flag, const int* jlo, const int* jn, cudaStream_t s) override {
        auto a = make_fwd_args<T>(g, in, out, kref, pose, jslot, flag, jlo, jn);
        if (this->rows_f == 1)
            launch_pdl(fwd_step_kernel<T, 3, HW, TX, TY, TZ>, this->fgrid, this->fthreads, smem_fwd, s, this->pdl, g, a);
        else if (this->rows_f == 8)
            launch_pdl(fwd3d_kernel<T, HW, 8>, this->fgrid, this->fthreads, smem3d_fwd<T>(), s, this->pdl, g, a);
        else if (this->rows_f == 16)
            launch_pdl(fwd3d_kernel<T, HW, 16>, this->fgrid, this->fthreads, smem3d_fwd<T>(), s, this->pdl, g, a);
        else if (this->rows_f == 32)
            launch_pdl(fwd3s_kernel<T, HW, 16, 8>, this->fgrid, this->fthreads, smem3s_fwd<T, 8>(), s, this->pdl, g, a);
        else if (this->rows_f == 64)
            launch_pdl(fwd3s_kernel<T, HW, 32, 8>, this->fgrid, this->fthreads, smem3s_fwd<T, 8>(), s, this->pdl, g, a);
        else if (this->rows_f == 96)
            launch_pdl(fwd3s_kernel<T, HW, 16, 16>, this->fgrid, this->fthreads, smem3s_fwd<T, 16>(), s, this->pdl, g, a);
        else if constexpr (kPair) {
            const bool v4 = g.n[0] % 4 == 0;
            if (this->rows_f == 128)
                launch_pdl(v4 ? fwd3p_kernel<HW, 16, true> : fwd3p_kernel<HW, 16, false>, this->fgrid, this->fthreads,
                           smem3p_fwd(), s, this->pdl, g, a);
            else
                launch_pdl(v4 ? fwd3p_kernel<HW, 32, true> : fwd3p_kernel<HW, 32, false>, this->fgrid, this->fthreads,
                           smem3p_fwd(), s, this->pdl, g, a);
        }
    }
    void adj(const Geom& g, const void* lam_in, void* lam_out, const void* prev, const void* cur, const void* kref,
             const Pose* pose, void* boxbuf, const void* fac, int src, cudaStream_t s) override {
        auto a = make_adj_args<T>(g, lam_in, lam_out, prev, cur, kref, pose, boxbuf, fac, src);
        if (this->rows_a == 1)
            launch_pdl(adj_step_kernel<T, 3, HW, TX, TY, TZ>, this->agrid, this->athreads, smem_adj, s, this->pdl, g, a);
        else if (this->rows_a == 8)
            launch_pdl(adj3d_kernel<T, HW, 8>, this->agrid, this->athreads, smem3d_adj<T>(), s, this->pdl, g, a);
        else if (this->rows_a == 16)
            launch_pdl(adj3d_kernel<T, HW, 16>, this->agrid, this->athreads, smem3d_adj<T>(), s, this->pdl, g, a);
        else if (this->rows_a == 32)
            launch_pdl(adj3s_kernel<T, HW, 16, 8>, this->agrid, this->athreads, smem3s_adj<T, 8>(), s, this->pdl, g, a);
        else if (this->rows_a == 64)
            launch_pdl(adj3s_kernel<T, HW, 32, 8>, this->agrid, this->athreads, smem3s_adj<T, 8>(), s, this->pdl, g, a);
        else if constexpr (kPair) {
            const bool v4 = g.n[0] % 4 == 0;
            if (this->rows_a == 128)
                launch_pdl(v4 ? adj3p_kernel<HW, 16, true> : adj3p_kernel<HW, 16, false>, this->agrid, this->athreads,
                           smem3p_adj(), s, this->pdl, g, a);
            else
                launch_pdl(v4 ? adj3p_kernel<HW, 32, true> : adj3p_kernel<HW, 32, false>, this->agrid, this->athreads,
                           smem3p_adj(), s, this->pdl, g, a);
        }
    }
};

}  // namespace lks
