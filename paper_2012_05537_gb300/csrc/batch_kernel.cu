// Persistent batched step kernels (FP32 storage, the generic kernel's tile body) and their
// host helpers: one launch advances every mesh of one order by one step.
#include "step_kernel.cuh"
#include "tables.h"

namespace sllbm {

namespace {

template <int P, int SH>
struct BatchShape;
template <> struct BatchShape<2, 0> { static constexpr int CX = 4, CY = 4, CZ = 2, NW = 16; };
template <> struct BatchShape<2, 1> { static constexpr int CX = 4, CY = 2, CZ = 2, NW = 16; };
template <> struct BatchShape<2, 2> { static constexpr int CX = 2, CY = 2, CZ = 1, NW = 8; };
template <> struct BatchShape<3, 0> { static constexpr int CX = 2, CY = 2, CZ = 2, NW = 16; };
template <> struct BatchShape<3, 1> { static constexpr int CX = 2, CY = 2, CZ = 1, NW = 16; };
template <> struct BatchShape<3, 2> { static constexpr int CX = 1, CY = 1, CZ = 1, NW = 8; };
template <> struct BatchShape<4, 0> { static constexpr int CX = 2, CY = 2, CZ = 1, NW = 16; };
template <> struct BatchShape<4, 1> { static constexpr int CX = 2, CY = 1, CZ = 1, NW = 16; };
template <> struct BatchShape<4, 2> { static constexpr int CX = 1, CY = 1, CZ = 1, NW = 8; };

template <int P, int SH>
auto kernel_of() {
    using B = BatchShape<P, SH>;
    return batch_step_kernel<float, P, B::CX, B::CY, B::CZ, B::NW>;
}

template <int P, int SH>
size_t smem_of() {
    using B = BatchShape<P, SH>;
    using SM = BatchSmem<float, P, B::CX, B::CY, B::CZ, B::NW>;
    static_assert(SM::bytes <= 227 * 1024, "shared memory budget");
    return SM::bytes;
}

template <int P, int SH>
int grid_t(int num_sms, long long items, int* grid) {
    auto k = kernel_of<P, SH>();
    const size_t smem = smem_of<P, SH>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BatchShape<P, SH>::NW * 32, smem);
    if (e != cudaSuccess) return SLLBM_ECUDA;
    long long g = static_cast<long long>(num_sms) * (per_sm > 0 ? per_sm : 1);
    if (g > items) g = items;
    *grid = static_cast<int>(g < 1 ? 1 : g);
    return SLLBM_OK;
}

// The velocity set in FP32, built once.
const Lattice<float>& lattice_f32() {
    static const Lattice<float> lat = [] {
        double xi[kQ][3], w[kQ];
        build_velocity_set(xi, w);
        Lattice<float> l;
        for (int i = 0; i < kQ; ++i) {
            for (int d = 0; d < 3; ++d) l.xi[i][d] = static_cast<float>(xi[i][d]);
            l.w[i] = static_cast<float>(w[i]);
        }
        return l;
    }();
    return lat;
}

template <int P, int SH>
int launch_t(const BatchJob* jobs, int njobs, const void* tabs, long long items, int parity, int grid,
             cudaStream_t st) {
    auto k = kernel_of<P, SH>();
    k<<<grid, BatchShape<P, SH>::NW * 32, smem_of<P, SH>(), st>>>(
        jobs, njobs, static_cast<const StepTables<float, P>*>(tabs), items, parity, lattice_f32());
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ECUDA;
}

template <int P>
void cells_t(int shape, int c[3]) {
    if (shape == 0) {
        c[0] = BatchShape<P, 0>::CX, c[1] = BatchShape<P, 0>::CY, c[2] = BatchShape<P, 0>::CZ;
    } else if (shape == 1) {
        c[0] = BatchShape<P, 1>::CX, c[1] = BatchShape<P, 1>::CY, c[2] = BatchShape<P, 1>::CZ;
    } else {
        c[0] = BatchShape<P, 2>::CX, c[1] = BatchShape<P, 2>::CY, c[2] = BatchShape<P, 2>::CZ;
    }
}

}  // namespace

void batch_tile_cells(int p, int shape, int cells[3]) {
    if (p == 2) cells_t<2>(shape, cells);
    else if (p == 3) cells_t<3>(shape, cells);
    else cells_t<4>(shape, cells);
}

size_t batch_tables_bytes(int p) {
    return p == 2 ? sizeof(StepTables<float, 2>) : p == 3 ? sizeof(StepTables<float, 3>) : sizeof(StepTables<float, 4>);
}

void batch_fill_tables(const sllbm_ctx* ctx, void* host_dst) {
    if (ctx->p == 2) fill_step_tables<float, 2>(ctx, static_cast<StepTables<float, 2>*>(host_dst));
    else if (ctx->p == 3) fill_step_tables<float, 3>(ctx, static_cast<StepTables<float, 3>*>(host_dst));
    else fill_step_tables<float, 4>(ctx, static_cast<StepTables<float, 4>*>(host_dst));
}

#define SLLBM_BATCH_DISPATCH(P, FN, ...)                        \
    switch (shape) {                                           \
    case 0: return FN<P, 0>(__VA_ARGS__);                      \
    case 1: return FN<P, 1>(__VA_ARGS__);                      \
    case 2: return FN<P, 2>(__VA_ARGS__);                      \
    }                                                          \
    return SLLBM_EINVAL

int batch_group_grid(int p, int shape, int num_sms, long long items, int* grid) {
    if (p == 2) { SLLBM_BATCH_DISPATCH(2, grid_t, num_sms, items, grid); }
    if (p == 3) { SLLBM_BATCH_DISPATCH(3, grid_t, num_sms, items, grid); }
    if (p == 4) { SLLBM_BATCH_DISPATCH(4, grid_t, num_sms, items, grid); }
    return SLLBM_EINVAL;
}

int launch_batch_group(int p, int shape, const BatchJob* jobs, int njobs, const void* tabs, long long items,
                       int parity, int grid, cudaStream_t stream) {
    if (p == 2) { SLLBM_BATCH_DISPATCH(2, launch_t, jobs, njobs, tabs, items, parity, grid, stream); }
    if (p == 3) { SLLBM_BATCH_DISPATCH(3, launch_t, jobs, njobs, tabs, items, parity, grid, stream); }
    if (p == 4) { SLLBM_BATCH_DISPATCH(4, launch_t, jobs, njobs, tabs, items, parity, grid, stream); }
    return SLLBM_EINVAL;
}

}  // namespace sllbm
