// D3Q15 engine (see lks_engine.cuh).
#pragma once

#include "lks_engine.cuh"
#include "lks_step3d.cuh"
#include "lks_step3s.cuh"
#include "lks_step3p.cuh"

#include <cstdint>
#include <cstring>
#include <type_traits>

namespace lks {

// Tensor map of a state (4 fields of N floats, field a at base + a N) as the 4-D tensor (x, y, z, field) with the
// plane-pair kernels' raw box (RX x RY x 1 x 4, i.e. one plane of all four fields).  False when the driver has no
// encoder or the layout does not qualify (n_x not a multiple of 4, base not 16-byte aligned): the kernels then copy
// with every thread.
inline bool pair_tensor_map(const Geom& g, const void* base, CUtensorMap& tm) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static const Encode enc = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return (Encode) nullptr;
        }
        return reinterpret_cast<Encode>(fn);
    }();
    static_assert(Pair3::RX == PairA3::RX && Pair3::RY == PairA3::RY, "one box for both kernels");
    std::memset(&tm, 0, sizeof(tm));
    if (enc == nullptr || g.n[0] % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t dim[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], 4};
    const cuuint64_t stride[3] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4, (cuuint64_t)g.N * 4};
    const cuuint32_t box[4] = {(cuuint32_t)Pair3::RX, (cuuint32_t)Pair3::RY, 1, 4};
    const cuuint32_t unit[4] = {1, 1, 1, 1};
    return enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dim, stride, box, unit,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// D3Q15 engine: rows = 1 selects the generic shared-memory tile kernels (32 x 4 x 4 nodes per block);
// rows = 8 or 16 the z-marching kernels with that many planes per block (32 x 8 columns); forward rows = 32,
// 64 the separable z-marching kernels with 16 or 32 planes per block (32 x 8 columns), forward rows = 96 the
// separable forward with 16 planes of 32 x 16 columns; FP32 rows = 128, 160 the plane-pair separable kernels (packed
// FP32x2, forward and adjoint) with 16 or 32 planes per block (32 x 8 columns), adjoint rows = 192 the plane-pair
// adjoint with 64 planes.
template <typename T, int HW>
struct Engine3D : EngineCommon<T, 3, HW> {
    static constexpr int TX = 32, TY = 4, TZ = 4;
    using TL = Tile<3, TX, TY, TZ>;
    static constexpr size_t smem_fwd = sizeof(T) * (4 * TL::S + 7 * TL::M);
    static constexpr size_t smem_adj = sizeof(T) * (4 * TL::S + 10 * TL::M);

    explicit Engine3D(const Geom& g) {
        if (const char* e = std::getenv("LKS_NO_TMA"); e != nullptr && *e != '\0' && std::atoi(e) != 0) tma_on = false;
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
            const int sm = (int)smem3p_fwd(), sa = (int)smem3p_adj();
            for (bool v4 : {true, false}) {
                LKS_CUDA(cudaFuncSetAttribute(fwd3p_fn<16>(v4), cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
                LKS_CUDA(cudaFuncSetAttribute(fwd3p_fn<32>(v4), cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
                LKS_CUDA(cudaFuncSetAttribute(adj3p_fn<16>(v4), cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
                LKS_CUDA(cudaFuncSetAttribute(adj3p_fn<32>(v4), cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
                LKS_CUDA(cudaFuncSetAttribute(adj3p_fn<64>(v4), cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
            }
        }
        this->alks_attr();
        set_rows(8, 8, g);
    }
    // the plane-pair kernels exist for the FP32 state only
    static constexpr bool kPair = std::is_same<T, float>::value;
    // planes per block of the plane-pair codes (0: not a plane-pair code of that kernel)
    static int pair_zb(int r, bool adj) {
        if (r == 128) return 16;
        if (r == 160) return 32;
        if (adj && r == 192) return 64;
        return 0;
    }
    template <int ZB>
    static void (*fwd3p_fn(bool v4))(Geom, FwdArgs<float>, CUtensorMap, int) {
        return v4 ? fwd3p_kernel<HW, ZB, true> : fwd3p_kernel<HW, ZB, false>;
    }
    template <int ZB>
    static void (*adj3p_fn(bool v4))(Geom, AdjArgs<float>, CUtensorMap, int) {
        return v4 ? adj3p_kernel<HW, ZB, true> : adj3p_kernel<HW, ZB, false>;
    }
    // tensor copies are used unless the environment of the context's creation turned them off (LKS_NO_TMA=1:
    // every block copies per thread)
    bool tma_on = true;
    // the plane-pair forward writes 1 / (1 + kappa) on the footprint box for the adjoint with the hat kernel, with
    // the arithmetic of box_fac below
    bool fwd_writes_fac() const override { return kPair && HW == 1 && pair_zb(this->rows_f, false) > 0; }
    void box_fac(const Geom& g, const Pose* poses, const void* kref, int n_first, int nsteps, void* out,
                 cudaStream_t s) override {
        if constexpr (kPair && HW == 1) {
            box_fac_hat3_kernel<<<dim3(nblk(g.Fbn, 256), nsteps, 1), 256, 0, s>>>(g, poses, (const float*)kref, n_first,
                                                                                 (float*)out);
            LKS_LAUNCHED();
        } else {
            EngineCommon<T, 3, HW>::box_fac(g, poses, kref, n_first, nsteps, out, s);
        }
    }
    // local sensitivities: the column kernel for the FP32 state and the hat kernel (discrete adjoint)
    void sens(const Geom& g, const Pose* poses, const void* kref, const void* boxbuf, long long bstride, int n_first,
              int nsteps, void* kbar, double* mslot, bool alks, cudaStream_t s) override {
        if constexpr (kPair && HW == 1) {
            if (!alks) {
                adj_sens_hat3_kernel<<<dim3(sens_blocks(g, alks), nsteps, 1), kSensHatNT, 0, s>>>(
                    g, poses, (const float*)kref, (const float*)boxbuf, bstride, n_first, (float*)kbar, mslot);
                LKS_LAUNCHED();
                return;
            }
        }
        EngineCommon<T, 3, HW>::sens(g, poses, kref, boxbuf, bstride, n_first, nsteps, kbar, mslot, alks, s);
    }
    // transposed mapping: the hat kernel's gather for the FP32 state (both sensitivity kernels leave kappa-bar = 0
    // outside the grid)
    void gather(const Geom& g, const Pose* poses, const void* kbar, int n_first, int nsteps, long long kstride,
                double* dkref, cudaStream_t s) override {
        if constexpr (kPair && HW == 1) {
            const long long nd = (long long)g.nde[0] * g.nde[1] * g.nde[2];
            design_gather_hat3_kernel<<<nblk(nd, kGatherHatNT), kGatherHatNT, 0, s>>>(g, poses, (const float*)kbar,
                                                                                   n_first, nsteps, kstride, dkref);
            LKS_LAUNCHED();
        } else {
            EngineCommon<T, 3, HW>::gather(g, poses, kbar, n_first, nsteps, kstride, dkref, s);
        }
    }
    int sens_blocks(const Geom& g, bool alks) const override {
        if (kPair && HW == 1 && !alks)
            return (int)(nblk((long long)g.Fb[0] * g.Fb[1], kSensHatNT) * nblk(g.Fb[2], kSensHatZC));
        return EngineCommon<T, 3, HW>::sens_blocks(g, alks);
    }
    std::vector<int> fwd_codes() const override {
        if (kPair) return {1, 8, 16, 32, 64, 96, 128, 160};
        return {1, 8, 16, 32, 64, 96};
    }
    std::vector<int> adj_codes() const override {
        if (kPair) return {1, 8, 16, 32, 64, 128, 160, 192};
        return {1, 8, 16, 32, 64};
    }
    static void geom(int r, bool adj, const Geom& g, dim3& th, dim3& tile, dim3& grid) {
        if (r == 1) {
            th = tile = dim3(TX, TY, TZ);
            grid = dim3(nblk(g.n[0], TX), nblk(g.n[1], TY), nblk(g.n[2], TZ));
        } else if (r >= 128) {  // plane-pair kernels: pair_zb planes of 32 x 8 columns
            const int zb = pair_zb(r, adj);
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
        auto okf = [](int r) { return r == 1 || r == 8 || r == 16 || r == 32 || r == 64 || r == 96 || (kPair && pair_zb(r, false) > 0); };
        auto oka = [](int r) { return r == 1 || r == 8 || r == 16 || r == 32 || r == 64 || (kPair && pair_zb(r, true) > 0); };
        if (!okf(rf) || !oka(ra)) return false;
        // the plane-pair kernels index in 32 bits: every field offset c N + i and box offset c Fbn + b must fit
        const bool small = 4 * g.N < (1LL << 31) && 6 * g.Fbn < (1LL << 31);
        if (!small && (rf >= 128 || ra >= 128)) return false;
        this->rows_f = rf;
        this->rows_a = ra;
        geom(rf, false, g, this->fthreads, this->ftile, this->fgrid);
        geom(ra, true, g, this->athreads, this->atile, this->agrid);
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
            a.fac_out = (float*)this->fac_out;
            CUtensorMap tm;
            const int ut = tma_on && pair_tensor_map(g, in, tm) ? 1 : 0;
            switch (pair_zb(this->rows_f, false)) {
                case 16: launch_pdl(fwd3p_fn<16>(v4), this->fgrid, this->fthreads, smem3p_fwd(), s, this->pdl, g, a, tm, ut); break;
                default: launch_pdl(fwd3p_fn<32>(v4), this->fgrid, this->fthreads, smem3p_fwd(), s, this->pdl, g, a, tm, ut); break;
            }
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
            CUtensorMap tm;
            const int ut = tma_on && pair_tensor_map(g, lam_in, tm) ? 1 : 0;
            switch (pair_zb(this->rows_a, true)) {
                case 16: launch_pdl(adj3p_fn<16>(v4), this->agrid, this->athreads, smem3p_adj(), s, this->pdl, g, a, tm, ut); break;
                case 64: launch_pdl(adj3p_fn<64>(v4), this->agrid, this->athreads, smem3p_adj(), s, this->pdl, g, a, tm, ut); break;
                default: launch_pdl(adj3p_fn<32>(v4), this->agrid, this->athreads, smem3p_adj(), s, this->pdl, g, a, tm, ut); break;
            }
        }
    }
};

}  // namespace lks
