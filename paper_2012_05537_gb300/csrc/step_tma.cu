// Host side of the TMA-fed persistent step kernel (step_tma.cuh) for FP32 storage and the
// 16-bit deviation storages: eligibility, the tensor maps of the source buffer, the
// per-velocity tables and the launch.
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "step_tma.cuh"

namespace sllbm {

namespace {

// Tile (in cells) of the TMA kernel per order: 8x8x4 nodes for p = 2 and p = 4, 6x9x3 for
// p = 3 (a tile of whole cells 9 nodes wide would not fit two tiles of streamed pairs in
// tensor memory; 9 rows of 3 planes keep 27 of the 32 lanes busy, and a mesh whose y cell
// count is not a multiple of 3 ends in a partial tile row).
template <int P>
struct TmaTile;
template <>
struct TmaTile<2> {
    static constexpr int CX = 4, CY = 4, CZ = 2;
};
template <>
struct TmaTile<3> {
    static constexpr int CX = 2, CY = 3, CZ = 1;
};
template <>
struct TmaTile<4> {
    static constexpr int CX = 2, CY = 2, CZ = 1;
};
// Stream warps (45 velocity pairs: one warp with 5, ten with 4).
template <int P>
constexpr int kConsumersFor = kStreamWarps;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int P>
void fill_tables_s(const sllbm_ctx* ctx, StepTablesS<P>* t) {
    for (int i = 0; i < kQ; ++i) {
        for (int d = 0; d < 3; ++d) {
            int kmn = ctx->dir[d].shift[i][0], kmx = kmn;
            for (int a = 0; a < P; ++a) {
                const int k = ctx->dir[d].shift[i][a];
                kmn = k < kmn ? k : kmn;
                kmx = k > kmx ? k : kmx;
            }
            t->kmin[i][d] = static_cast<signed char>(kmn);
            t->span[i][d] = static_cast<signed char>(kmx - kmn);
            for (int a = 0; a < P; ++a) {
                t->kc[i][d][a] = static_cast<signed char>(ctx->dir[d].shift[i][a] - kmn);
                for (int j = 0; j <= P; ++j) {
                    t->lw[i][d][a][j] = static_cast<float>(ctx->dir[d].weight[i][a][j]);
                }
            }
            t->xi[i][d] = static_cast<float>(ctx->xi[i][d]);
        }
        t->w[i] = static_cast<float>(ctx->w[i]);
    }
}

template <int P>
bool tma_eligible_p(const sllbm_ctx* c) {
    using T = TmaTile<P>;
    if (c->cells[0] % T::CX != 0 || c->cells[2] % T::CZ != 0) return false;
    if (P != 3 && c->cells[1] % T::CY != 0) return false;
    // the passes are compiled per first local node of the upper departure cell: the shifts of
    // a cell's local nodes must not decrease with the node (they do not: the support points
    // are ordered, and so are their departure points)
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < kQ; ++i)
            for (int a = 1; a < P; ++a)
                if (c->dir[d].shift[i][a] < c->dir[d].shift[i][a - 1]) return false;
    return true;
}

// Builds (or reuses) the TMA descriptors of a source buffer: the buffer seen as a 4D tensor
// [45][Nz][Ny][X] (f_i, g_i interleaved along x): FP32 elements with X = 2*Nx for FP32
// storage, one 32-bit element per 16-bit (f, g) pair with X = Nx otherwise; one descriptor per
// box shape (span 0 or 1 of the departure cells in x, y, z).  Out-of-domain elements read as
// zero.
template <typename S, int P>
int tensor_maps_for(sllbm_ctx* ctx, const void* src, TmaMaps* out) {
    using T = TmaTile<P>;
    using G = TmaGeom<S, P, T::CX, T::CY, T::CZ>;
    constexpr cuuint64_t XM = G::kF32 ? 2 : 1;  // elements per pair
    const int k = (src == ctx->buf[0]) ? 0 : 1;
    if (ctx->tmap_src[k] != src) {
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (enc == nullptr) return SLLBM_ECUDA;
        const cuuint64_t nx = XM * ctx->N[0];
        cuuint64_t gdim[4] = {nx, static_cast<cuuint64_t>(ctx->N[1]), static_cast<cuuint64_t>(ctx->N[2]),
                              static_cast<cuuint64_t>(kQ)};
        cuuint64_t gstride[3] = {nx * 4, nx * ctx->N[1] * 4, nx * ctx->N[1] * ctx->N[2] * 4};
        cuuint32_t estride[4] = {1, 1, 1, 1};
        const CUtensorMapDataType dt = G::kF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
        for (int shape = 0; shape < 8; ++shape) {
            CUtensorMap map;
            cuuint32_t box[4] = {static_cast<cuuint32_t>(XM * G::xpairs_s(shape & 1)),
                                 static_cast<cuuint32_t>(G::rows((shape >> 1) & 1)),
                                 static_cast<cuuint32_t>(G::planes((shape >> 2) & 1)), 1u};
            CUresult r = enc(&map, dt, 4, const_cast<void*>(src), gdim, gstride, box, estride,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                ctx->tmap_src[k] = nullptr;
                return SLLBM_ECUDA;
            }
            std::memcpy(ctx->tmap[k][shape], &map, sizeof(map));
        }
        ctx->tmap_src[k] = src;
    }
    std::memcpy(out, ctx->tmap[k], sizeof(TmaMaps));
    return SLLBM_OK;
}

// Per-velocity coefficients of the Prandtl term (see PrTablesS), from the velocity set in FP64.
void fill_pr_tables(const sllbm_ctx* ctx, PrTablesS* pt) {
    for (int i = 0; i < kQ; ++i) {
        const double x = ctx->xi[i][0], y = ctx->xi[i][1], z = ctx->xi[i][2];
        const double a[10] = {x * x * x - 3 * x,     y * y * y - 3 * y,     z * z * z - 3 * z,     3 * x * x * y - 3 * y,
                              3 * x * x * z - 3 * z, 3 * y * y * x - 3 * x, 3 * y * y * z - 3 * z, 3 * z * z * x - 3 * x,
                              3 * z * z * y - 3 * y, 6 * x * y * z};
        for (int k = 0; k < 10; ++k) pt->a[i][k] = static_cast<float>(a[k] / 6.0);
    }
}

template <typename S, int P, bool PR, bool KC>
int launch_tma(sllbm_ctx* ctx, const void* src, void* dst) {
    using T = TmaTile<P>;
    constexpr int kConsumers = kConsumersFor<P>;
    using SM = TmaSmem<S, P, T::CX, T::CY, T::CZ, kConsumers, PR, KC>;
    static_assert(SM::bytes <= kSmemBudget, "shared memory budget");
    using Tab = StepTablesS<P>;
    if (ctx->step_blob == nullptr || ctx->step_blob_size != sizeof(Tab) + 1) {
        std::free(ctx->step_blob);
        ctx->step_blob = static_cast<unsigned char*>(std::malloc(sizeof(Tab)));
        if (ctx->step_blob == nullptr) return SLLBM_ENOMEM;
        ctx->step_blob_size = sizeof(Tab) + 1;  // +1 keeps it distinct from the generic tables
        fill_tables_s<P>(ctx, reinterpret_cast<Tab*>(ctx->step_blob));
    }
    TmaMaps maps;
    int rc = tensor_maps_for<S, P>(ctx, src, &maps);
    if (rc != SLLBM_OK) return rc;
    StepArgs args;
    fill_step_args(ctx, src, dst, &args);
    PrTablesS prt;
    if (PR) {
        fill_pr_tables(ctx, &prt);
    } else {
        std::memset(&prt, 0, sizeof(prt));
    }
    auto k = step_tma_kernel<S, P, T::CX, T::CY, T::CZ, kConsumers, PR, KC>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
    // all z-tiles, or the part of a slab's tiles its split step asks for (one launch per range)
    int ranges[2][2];
    const int nr = slab_tile_ranges(ctx, T::CZ, ranges);
    for (int q = 0; q < nr && err == cudaSuccess; ++q) {
        args.tz_begin = ranges[q][0];
        args.cells[2] = (ranges[q][1] - ranges[q][0]) * T::CZ;
        const int ntiles =
            (ctx->cells[0] / T::CX) * ((ctx->cells[1] + T::CY - 1) / T::CY) * (ranges[q][1] - ranges[q][0]);
        if (ntiles <= 0) continue;
        const int grid = ntiles < ctx->num_sms ? ntiles : ctx->num_sms;
        k<<<grid, kWarps * 32, SM::bytes, ctx->stream>>>(maps, args, *reinterpret_cast<const Tab*>(ctx->step_blob), prt);
        err = cudaGetLastError();
        ctx->launches += 1;
    }
    if (err != cudaSuccess) {
        ctx->last_err = static_cast<int>(err);
        return SLLBM_ECUDA;
    }
    return SLLBM_OK;
}

}  // namespace

bool tma_step_eligible(const sllbm_ctx* c) {
    const int st = c->prm.storage;
    if (st != SLLBM_F32 && st != SLLBM_F16DEV && st != SLLBM_BF16DEV) return false;
    // (the Prandtl term with FP32 storage only; compensated moment sums without it)
    if ((c->prm.pr_correction && (st != SLLBM_F32 || c->compensated)) || !c->prm.collide) return false;
    // TMA rows start on 16 bytes: x a multiple of 2 (FP32) or 4 (16-bit) pairs, so a row
    // of the mesh must be one too
    if (c->N[0] % (st == SLLBM_F32 ? 2 : 4) != 0 || c->num_sms <= 0) return false;
    if (tensor_map_encoder() == nullptr) return false;
    switch (c->p) {
    case 2: return tma_eligible_p<2>(c);
    case 3: return tma_eligible_p<3>(c);
    case 4: return tma_eligible_p<4>(c);
    }
    return false;
}

namespace {
template <typename S, bool PR, bool KC = false>
int launch_tma_for(sllbm_ctx* ctx, const void* src, void* dst) {
    switch (ctx->p) {
    case 2: return launch_tma<S, 2, PR, KC>(ctx, src, dst);
    case 3: return launch_tma<S, 3, PR, KC>(ctx, src, dst);
    case 4: return launch_tma<S, 4, PR, KC>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}
}  // namespace

int launch_step_tma(sllbm_ctx* ctx, const void* src, void* dst) {
    switch (ctx->prm.storage) {
    case SLLBM_F32:
        if (ctx->prm.pr_correction) return launch_tma_for<float, true>(ctx, src, dst);
        return ctx->compensated ? launch_tma_for<float, false, true>(ctx, src, dst)
                                : launch_tma_for<float, false>(ctx, src, dst);
    case SLLBM_F16DEV:
        return ctx->compensated ? launch_tma_for<__half, false, true>(ctx, src, dst)
                                : launch_tma_for<__half, false>(ctx, src, dst);
    case SLLBM_BF16DEV:
        return ctx->compensated ? launch_tma_for<__nv_bfloat16, false, true>(ctx, src, dst)
                                : launch_tma_for<__nv_bfloat16, false>(ctx, src, dst);
    }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
