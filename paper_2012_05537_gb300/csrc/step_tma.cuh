// Fused SLLBM step for FP32 and 16-bit deviation storage on sm_100-family GPUs: TMA-fed,
// warp-specialised, persistent, with the streamed populations parked in tensor memory.  Same
// arithmetic as step_kernel.cuh (Eq. interpolation, Eq. moments, Eq. discreteEquilibrium,
// Eq. LBM), organised for GB300:
//
//  * One persistent CTA per SM walks tiles of CX x CY x CZ cells (TX x TY x TZ nodes).
//  * A producer warp loads, for every velocity i of a tile, the source box of the pair
//    (f_i, g_i) -- the tile translated by the departure cell shift, plus the cells and the
//    shared face the departure points reach; a box is one cell shorter in each direction
//    where all local nodes depart from the same cell -- into a ring of shared memory that
//    is allocated in 128-byte units and reclaimed in order: one 4D TMA load
//    (cp.async.bulk.tensor) when the box lies inside the periodic domain; when it crosses
//    the boundary, one TMA load per periodic image it overlaps, back to back (zero-filled
//    outside the domain, summed by the consumer on its first pass), or 16-byte cp.async
//    copies from the wrapped positions when that takes too many images.  Items are handed
//    over through a ring of 32 descriptors: full/empty mbarriers (transaction counts) and
//    an item table entry that tells the consumers where the item's box sits.
//  * 11 stream warps own 4 or 5 velocity pairs each.  For a pair they run the z and y
//    Lagrange passes in place in the box (each lane owns whole columns; a 16-bit box is
//    widened to FP32 by the z pass, into the warp's scratch) and the x pass into registers
//    (lane = one x-row of the tile), then release the box.  f_i and g_i share weights and
//    positions, so every FMA is a packed FP32x2 FMA.  The streamed (f_i, g_i) of the lane's
//    TX nodes go to the lane's row of tensor memory (tcgen05.st), in one of two buffers per
//    tile parity.
//  * Four epilogue warps, one per tensor-memory lane quarter, take a tile's buffer once the
//    quarter's stream warps are done with it: per-node moment sums of the quarter's pairs,
//    the sum over the quarters in a fixed order (deterministic), rho, u, T, omega and the
//    shell coefficients of the quartic equilibrium (each epilogue warp a quarter of the
//    nodes), then the collision of the quarter's pairs and 16- or 8-byte stores (f_i and g_i
//    interleaved).  Meanwhile the stream warps fill the other buffer: streaming never
//    waits for the collision.
//  * With the quasi-equilibrium Prandtl term (App. D, FP32 storage) the epilogue warps also
//    form the centred third moment of the streamed f per node, in a second pass over their
//    buffer (two rounds of five components, the quarters summed through shared memory), and
//    add the term to the collision.
//  * With compensated moment sums (KC; FP32 arithmetic, without the Prandtl term) each
//    epilogue warp keeps a two-sum running sum and its error per moment and node, and the
//    quarters' sums and errors are merged in the same compensated way, so a moment carries
//    about one FP32 rounding.
//  * Every mbarrier wait is bounded; on expiry the kernel raises an error flag, the stream
//    and epilogue warps leave (and free the tensor memory) and the producer waits (bounded)
//    for its copies in flight before returning.
#pragma once

#include <cuda.h>

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "collide.cuh"
#include "compsum.cuh"
#include "packed.cuh"
#include "sllbm_internal.h"

namespace sllbm {

// Per-velocity tables; passed by value, then copied once per CTA into shared memory so that
// every lane reads the (warp-uniform) entries of its pair with broadcast loads.
template <int P>
struct StepTablesS {
    float lw[kQ][3][P][P + 1];  // Lagrange weights per (velocity, direction, local node)
    float xi[kQ][3];
    float w[kQ];
    signed char kc[kQ][3][P];   // departure cell shift minus kmin (0 or 1)
    signed char kmin[kQ][3];
    signed char span[kQ][3];
};

// Coefficients of the quasi-equilibrium Prandtl term per velocity (App. D): with Qbar the
// centred third moment of the streamed f and q_a = sum_b Qbar_abb, f*_i / w_i =
// (Qbar : H3(xi_i)) / 6 = sum_k a[i][k] Qbar_k over Qbar_xxx, Qbar_yyy, Qbar_zzz, Qbar_xxy,
// Qbar_xxz, Qbar_yyx, Qbar_yyz, Qbar_zzx, Qbar_zzy, Qbar_xyz, with a = (x^3 - 3x, y^3 - 3y,
// z^3 - 3z, 3x^2y - 3y, 3x^2z - 3z, 3y^2x - 3x, 3y^2z - 3z, 3z^2x - 3x, 3z^2y - 3y, 6xyz) / 6.
struct PrTablesS {
    float a[kQ][10];
};

// Box and tile geometry for storage type S (float: f and g themselves; __half or
// __nv_bfloat16: their deviations, see storage.cuh).  A box is held in the ring as stored
// (rows of pairs from an x that TMA can address: a multiple of AL pairs, 16 bytes); the
// passes run in FP32 on rows of pairs from an even x (in place in the ring for FP32, in the
// stream warp's scratch otherwise).
template <typename S, int P, int CX, int CY, int CZ>
struct TmaGeom {
    static constexpr bool kF32 = sizeof(S) == 4;
    static constexpr int PB = 2 * static_cast<int>(sizeof(S));  // bytes of one stored (f, g) pair
    static constexpr int AL = 16 / PB;                           // pairs per 16 bytes
    static constexpr int TX = CX * P, TY = CY * P, TZ = CZ * P;
    static constexpr int TILE = TX * TY * TZ;
    static constexpr int ROWS = TY * TZ;  // x-rows of a tile, one per lane
    static constexpr int BX = (CX + 1) * P + 1, BY = (CY + 1) * P + 1, BZ = (CZ + 1) * P + 1;
    static constexpr int BXP = ((BX + 1) + 1) / 2 * 2;  // FP32 pairs per box row: even start + offset
    static constexpr int PLANE = BY * BXP;              // float2 per box plane
    static constexpr int BOX = BZ * PLANE;              // float2 per box
    // A velocity whose P local nodes all depart from the same cell in a direction (span 0)
    // needs one cell less of the box in that direction.  Box extents per span:
    static constexpr int BX0 = CX * P + 1, BY0 = CY * P + 1, BZ0 = CZ * P + 1;
    static constexpr int BXP0 = ((BX0 + 1) + 1) / 2 * 2;
    // stored pairs per ring row (from the x rounded down to a multiple of AL)
    static constexpr int BXS = (BX + AL - 1 + AL - 1) / AL * AL, BXS0 = (BX0 + AL - 1 + AL - 1) / AL * AL;
    __host__ __device__ static constexpr int xpairs(int span) { return span ? BXP : BXP0; }
    __host__ __device__ static constexpr int xpairs_s(int span) { return span ? BXS : BXS0; }
    __host__ __device__ static constexpr int rows(int span) { return span ? BY : BY0; }
    __host__ __device__ static constexpr int planes(int span) { return span ? BZ : BZ0; }
    // bytes of a stored box of shape sx + 2 sy + 4 sz, and the 128-byte ring units one piece takes
    __host__ __device__ static constexpr int box_bytes(int shape) {
        return xpairs_s(shape & 1) * rows((shape >> 1) & 1) * planes((shape >> 2) & 1) * PB;
    }
    __host__ __device__ static constexpr int piece_units(int shape) { return (box_bytes(shape) + 127) / 128; }
    static constexpr int SLOT_BYTES = (BXS * BY * BZ * PB + 127) / 128 * 128;
    // FP32 working copy of a 16-bit box after the z pass (TZ planes), per stream warp
    static constexpr int SCRATCH_F2 = kF32 ? 0 : TZ * BY * BXP;
    // tensor-memory columns per streamed pair (2 TX used; a multiple of 16 keeps every
    // tcgen05 access aligned to its width)
    static constexpr int PCS = (2 * TX + 15) / 16 * 16;
    static_assert(ROWS <= 32, "one x-row per lane");
    static_assert(BXP % 2 == 0 && BXP >= BX + 1 && BXP0 % 2 == 0 && BXP0 >= BX0 + 1, "pass rows start on an even pair");
    static_assert(BXS % AL == 0 && BXS >= BX + AL - 1 && BXS0 % AL == 0 && BXS0 >= BX0 + AL - 1, "TMA rows");
    // a 16-bit row is read from its even pair at or below the first used one (AL - 2 at most
    // above the row start) for BXP pairs
    static_assert(kF32 || (AL - 2 + BXP <= BXS && AL - 2 + BXP0 <= BXS0), "z pass reads stay in the row");
    static_assert(TX == 8 || TX == 6, "tensor-memory row layout and node shares of the epilogue warps");
};

// One TMA descriptor per box shape (span 0/1 in x, y, z: index sx + 2 sy + 4 sz) of a source
// buffer, passed to the kernel as one parameter block.
struct TmaMaps {
    CUtensorMap m[8];
};

constexpr int kNParams = 18;  // rho, ux, uy, uz, gT, omega, c0[4], c1[4], c2[4]

// Warp roles.  A warp's SM sub-partition is its index mod 4, and so is the tensor-memory lane
// quarter it may touch.  Warp 1 is the producer; warps 12..15 are the epilogue warps, one per
// quarter; the other 11 are stream warps, three in quarters 0, 2 and 3 and two (5, 9) in
// quarter 1, next to the producer.  Stream warp c (c = 0..10, warp 5 first) streams the pairs
// j = c, c + 11, c + 22, ... (five for c = 0, four for the others), so the quarters hold
// 12, 9, 12 and 12 pairs: every sub-partition has work, and the one with the producer the
// least.  (Nine stream warps in quarters 0, 2, 3 with 15 pairs each and sub-partition 1 left
// to the producer alone measured 3 % slower at p = 4 and 7-9 % slower at p = 3.)
constexpr int kWarps = 16;
constexpr int kEpilogueWarps = 4;
constexpr int kStreamWarps = 11;
constexpr int kMaxPairsPerWarp = (kQ + kStreamWarps - 1) / kStreamWarps;  // 5
constexpr int NPROD = 1;    // producers
constexpr int IPP = kQ;     // items per tile and producer
__host__ __device__ constexpr bool is_producer_warp(int w) { return w == 1; }
__host__ __device__ constexpr int producer_index(int) { return 0; }
__host__ __device__ constexpr bool is_stream_warp(int w) { return w < 12 && w != 1; }
__host__ __device__ constexpr int stream_index(int w) { return w == 5 ? 0 : (w == 0 ? 1 : (w < 5 ? w : w - 1)); }
// velocity pairs of stream warp c, and the k-th of them
__host__ __device__ constexpr int pairs_of(int c) { return (kQ - c + kStreamWarps - 1) / kStreamWarps; }
__host__ __device__ constexpr int pair_of(int c, int k) { return c + kStreamWarps * k; }
__host__ __device__ constexpr bool is_epilogue_warp(int w) { return w >= 12; }
__host__ __device__ constexpr int epilogue_index(int w) { return w - 12; }
static_assert(pairs_of(0) == kMaxPairsPerWarp && pairs_of(1) == 4 && pairs_of(10) == 4, "pair split");
// A source box that crosses the periodic boundary is loaded as one TMA box per periodic image
// it overlaps (zero outside the domain), at most kMaxPieces of them, back to back in the ring;
// boxes with more images (meshes not much larger than a tile), or whose images would not fit
// in the producer's part of the ring, take the cp.async path.
constexpr int kMaxPieces = 8;
// Items in flight at most: the descriptor ring (full/empty mbarriers, item table entry and
// ring offset per item; a power of two).
constexpr int kItems = 32;
constexpr size_t kSmemBudget = 227 * 1024;
static_assert((kItems & (kItems - 1)) == 0, "item table size");

template <typename S, int P, int CX, int CY, int CZ, int NC, bool PR = false, bool KC = false>
struct TmaSmem {
    using G = TmaGeom<S, P, CX, CY, CZ>;
    // every region starts on a 128-byte boundary (TMA destinations, float4 and mbarrier
    // alignment)
    static constexpr size_t round128(size_t b) { return (b + 127) / 128 * 128; }
    // per-node parameters of the collision: rho, ux, uy, uz, gT, omega, c0[4], c1[4], c2[4]
    // (FP32 storage); rho, ux, uy, uz, omega, rho - rho0, (2C_v-D) T rho, (2C_v-D)((T - T0) rho
    // + T0 (rho - rho0)), c0[4] - 1, c1[4], c2[4] (deviation storage)
    static constexpr int kNPar = G::kF32 ? kNParams : kNParams + 2;
    // the per-quarter moment sums (4 quarters x 5, then with compensated sums their 4 x 5 error
    // terms) and the per-node parameters share one region: an epilogue warp reads the sums of
    // exactly the node columns whose parameters it writes
    static constexpr int kSumRows = KC ? 2 * 4 * 5 : 4 * 5;
    static constexpr int kShared = kSumRows > kNPar ? kSumRows : kNPar;
    static constexpr size_t partials = round128(size_t(kShared) * G::TX * 32 * sizeof(float));
    static constexpr size_t params = 0;
    static constexpr size_t tables = round128(sizeof(StepTablesS<P>));
    // per producer: full[kItems], empty[kItems] mbarriers and the item table (one word per
    // entry: item number, ring offset and piece count); tmem_full[4][2], tmem_empty[4][2]
    // mbarriers; per producer the ring offsets of its items in flight; flags
    static constexpr size_t bars =
        (size_t(NPROD) * 3 * kItems + 16) * sizeof(uint64_t) + size_t(NPROD) * kItems * sizeof(int) + 16;
    static constexpr size_t bars_padded = round128(bars);
    static constexpr int woff_n = G::BZ + G::BY + G::BXS / G::AL;  // wrapped-offset table per producer
    static constexpr size_t woff = round128(size_t(NPROD) * woff_n * sizeof(long long));
    static constexpr size_t stage = size_t(kEpilogueWarps) * 32 * 64;  // one pair's 32 rows per epilogue warp
    static constexpr size_t scratch = round128(size_t(NC) * G::SCRATCH_F2 * 8);  // 16-bit storage only
    // Prandtl term only: the quarters' partial sums of five components of the centred third
    // moment (4 x 5 rows), the ten components per node (10 rows) and the per-velocity
    // coefficients of the term (kQ x 10)
    static constexpr int kQRows = 30;
    static constexpr size_t qreg = PR ? round128((size_t(kQRows) * G::TX * 32 + size_t(kQ) * 10) * sizeof(float)) : 0;
    static constexpr size_t fixed =
        partials + params + tables + bars_padded + woff + stage + scratch + qreg + 128;  // +128: base alignment
    // the box ring takes the rest, in 128-byte units
    static constexpr int ring_units = static_cast<int>((kSmemBudget - fixed) / 128);
    static constexpr size_t ring = size_t(ring_units) * 128;
    static constexpr size_t bytes = ring + fixed;
    static_assert(ring_units / NPROD >= G::SLOT_BYTES / 128, "each producer's ring holds the largest box");
};

// Tensor-memory columns: a stream warp's lane keeps up to NPW pairs x 2*TX floats per tile (PCS
// columns per pair); stream warps w, w+4, w+8 share a 32-lane quarter (the quarter a warp may
// touch is fixed by w % 4; warp w's columns are the (w / 4)-th share); each quarter holds two
// tiles (buffers).
template <int PCS, int NPW, int NC>
struct TmemCols {
    static constexpr int per_warp = NPW * PCS;
    static constexpr int per_buf = ((NC + 3) / 4) * per_warp;
    static constexpr int per_quarter = 2 * per_buf;
    static constexpr int alloc = per_quarter <= 32 ? 32 : per_quarter <= 64 ? 64 : per_quarter <= 128 ? 128
                               : per_quarter <= 256 ? 256 : 512;
    static_assert(per_quarter <= 512, "tensor memory columns");
};

// compile-time integer as a value (selects a pass variant in a generic lambda)
template <int V>
struct IntC {
    static constexpr int value = V;
};

// ------------------------------------------------------------------ PTX helpers
// One stored 16-bit (f, g) pair (a 32-bit word) as two floats, and two floats rounded to one.
template <typename S>
__device__ __forceinline__ float2 widen_pair(uint32_t w) {
    if constexpr (std::is_same<S, __half>::value) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
}

template <typename S>
__device__ __forceinline__ uint32_t narrow_pair(float f, float g) {
    uint32_t w;
    if constexpr (std::is_same<S, __half>::value) {
        const __half2 h = __floats2half2_rn(f, g);
        memcpy(&w, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f, g);
        memcpy(&w, &h, 4);
    }
    return w;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Non-blocking test: has the phase with this parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// One poll: the thread may sleep until the phase completes, but at most ~1 us (the
// suspend-time hint).
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded waits give up after limit_ns of wall time (read from the global timer; the step
// arguments carry the limit of the consumers' and the producer's waits, 2 s unless
// sllbm_set_wait_limit changed it), or after kWaitPolls polls should that timer not advance,
// or as soon as another warp raised the CTA abort flag; the warp that gives up raises the
// abort flag and the global error bit.  The producer's drain of its copies in flight always
// waits up to kWaitNs.
constexpr uint64_t kWaitNs = kDefaultWaitNs;
constexpr uint32_t kWaitPolls = 1u << 26;

__device__ __forceinline__ bool wait_give_up(volatile int* abort_flag, int* err_flag) {
    *abort_flag = 1;
    if (err_flag != nullptr) atomicOr(err_flag, 2);
    return false;
}

// Bounded wait for the phase `parity` of an mbarrier.  try_wait suspends the thread until the
// phase completes (or the hint expires), so the loop does not spin on the issue slots.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                                  int* err_flag, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < kWaitPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7u) == 0) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    return wait_give_up(abort_flag, err_flag);
}

// Bounded wait until the high half of a shared-memory word (written with one 64-bit store)
// reaches `want`; returns the low half (0 if the wait gave up, same give-up rules).  Short
// sleeps between polls leave the issue slots to the warps doing work.
__device__ __forceinline__ uint32_t wait_item_bounded(volatile unsigned long long* word, uint32_t want,
                                                      volatile int* abort_flag, int* err_flag, uint64_t limit_ns) {
    unsigned long long v = *word;
    if (static_cast<uint32_t>(v >> 32) == want) return static_cast<uint32_t>(v);
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < kWaitPolls; ++it) {
        __nanosleep(32);
        v = *word;
        if (static_cast<uint32_t>(v >> 32) == want) return static_cast<uint32_t>(v);
        if ((it & 7u) == 0) {
            if (*abort_flag) return 0;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    wait_give_up(abort_flag, err_flag);
    return 0;
}

// floor(a / n) for n > 0; the usual cases (|a| < 2n) without a division
__device__ __forceinline__ int floor_div(int a, int n) {
    if (a >= 0 && a < n) return 0;
    if (a < 0 && a >= -n) return -1;
    if (a >= n && a < 2 * n) return 1;
    const int q = a / n;
    return (a % n != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// The mbarrier receives one arrival once all earlier cp.async copies of the thread landed.
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier 1 over the stream and epilogue warps with an OR vote (all threads get the
// same answer).
__device__ __forceinline__ int consumer_barrier_or(int v, int nthreads) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred pin, pout;\n\tsetp.ne.u32 pin, %1, 0;\n\t"
        "barrier.cta.red.or.pred pout, 1, %2, pin;\n\tselp.u32 %0, 1, 0, pout;\n\t}"
        : "=r"(out)
        : "r"(v), "r"(nthreads)
        : "memory");
    return static_cast<int>(out);
}

// Named barrier 2 over the epilogue warps, with an OR vote.
__device__ __forceinline__ int epilogue_barrier_or(int v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred pin, pout;\n\tsetp.ne.u32 pin, %1, 0;\n\t"
        "barrier.cta.red.or.pred pout, 2, %2, pin;\n\tselp.u32 %0, 1, 0, pout;\n\t}"
        : "=r"(out)
        : "r"(v), "r"(kEpilogueWarps * 32)
        : "memory");
    return static_cast<int>(out);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit tensor-memory columns of the calling thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t ta, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(ta),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
        : "memory");
}

// 8 and 4 consecutive columns (the column address a multiple of 8 and 4).
__device__ __forceinline__ void tmem_st8(uint32_t ta, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t ta, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(ta), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "r"(ta)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t ta, float* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(ta)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t ta, float* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(ta)
                 : "memory");
}

// 2*TX floats (TX = 8 or 6) of one pair at column ta (a multiple of 16).
template <int TX>
__device__ __forceinline__ void tmem_store_row(uint32_t ta, const float* v) {
    if constexpr (TX == 8) {
        tmem_st16(ta, v);
    } else {
        static_assert(TX == 6, "row widths");
        tmem_st8(ta, v);
        tmem_st4(ta + 8, v + 8);
    }
}

// (the caller waits with tcgen05.wait::ld before using v)
template <int TX>
__device__ __forceinline__ void tmem_load_row(uint32_t ta, float* v) {
    if constexpr (TX == 8) {
        tmem_ld16(ta, v);
    } else {
        static_assert(TX == 6, "row widths");
        tmem_ld8(ta, v);
        tmem_ld4(ta + 8, v + 8);
    }
}

// 2*CH floats of one pair at column ta: CH = 4 nodes (half of an 8-node row), or a whole
// 6-node row
template <int CH>
__device__ __forceinline__ void tmem_load_nodes(uint32_t ta, float* v) {
    if constexpr (CH == 4) {
        tmem_ld8(ta, v);
    } else {
        tmem_load_row<CH>(ta, v);
    }
}

// Visiting order of the tiles: slabs of kBlockZ tile layers; in a slab, blocks of kBlockXY x
// kBlockXY tile columns (row by row); in a block, z-, y-, then x-slowest.  Consecutive tiles
// (the CTAs of one wave) thus cover a compact region whose source boxes overlap in L2, rather
// than one thin layer of tiles whose z-halo (a box is 2.25 cells deep for a 1-cell tile) is
// read again by the next wave.  Edge slabs, rows and blocks are simply thinner.  Returns the
// tile's (x, y, z) tile coordinates.  (Columns 8 tiles deep measured best with the
// four-quarter warp layout: 1.3 % faster than 16 at p = 4 on 128^3 nodes, as fast or faster
// at p = 3, and 4, 32 or 64 deep or 2x2-column blocks slower; with the earlier layout 16 had
// been best, within a few per cent of 2x2x16, 2x2x32 and 4x4x8 blocks.)
#ifndef SLLBM_TILE_BLOCK_XY
#define SLLBM_TILE_BLOCK_XY 1
#endif
#ifndef SLLBM_TILE_BLOCK_Z
#define SLLBM_TILE_BLOCK_Z 8
#endif
constexpr int kBlockXY = SLLBM_TILE_BLOCK_XY, kBlockZ = SLLBM_TILE_BLOCK_Z;
__device__ __forceinline__ void tile_coords(int t, int ntx, int nty, int ntz, int* tc) {
    const int slab = t / (ntx * nty * kBlockZ);
    const int bz = min(kBlockZ, ntz - slab * kBlockZ);
    int u = t - slab * ntx * nty * kBlockZ;
    const int yb = u / (ntx * kBlockXY * bz);
    const int by = min(kBlockXY, nty - yb * kBlockXY);
    u -= yb * ntx * kBlockXY * bz;
    const int xb = u / (kBlockXY * by * bz);
    const int bx = min(kBlockXY, ntx - xb * kBlockXY);
    u -= xb * kBlockXY * by * bz;
    tc[0] = xb * kBlockXY + u % bx;
    tc[1] = yb * kBlockXY + (u / bx) % by;
    tc[2] = slab * kBlockZ + u / (bx * by);
}

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------------------ kernel
template <typename S, int P, int CX, int CY, int CZ, int NC, bool PR, bool KC>
__global__ void __launch_bounds__(kWarps * 32, 1)
    step_tma_kernel(const __grid_constant__ TmaMaps maps, const StepArgs a,
                    const __grid_constant__ StepTablesS<P> tpar, const __grid_constant__ PrTablesS prt) {
    using G = TmaGeom<S, P, CX, CY, CZ>;
    using SM = TmaSmem<S, P, CX, CY, CZ, NC, PR, KC>;
    static_assert(!(KC && PR), "compensated sums without the Prandtl term");
    static_assert(!PR || G::kF32, "the Prandtl term runs with FP32 storage");
    constexpr int NPW = kMaxPairsPerWarp;  // velocity pairs per stream warp, at most
    using TC = TmemCols<G::PCS, NPW, NC>;
    // (x in the tensor maps counts floats for FP32 storage, (f, g) pairs for 16-bit storage)
    constexpr int XM = G::kF32 ? 2 : 1;
    // p = 3 tiles are 3 cells high: the last tile row of a mesh whose y cell count is not a
    // multiple of 3 is partial (its missing x-rows are computed from in-box data and dropped)
    constexpr bool kRaggedY = CY == 3;
    constexpr uint32_t KM = kItems - 1;
    constexpr int NE = kEpilogueWarps;
    static_assert(NC == kStreamWarps && NE == 4, "warp roles");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    unsigned char* ringb = base;  // the box ring, in 128-byte units
    float* part = reinterpret_cast<float*>(base + SM::ring);
    float* prm = part;  // (the same region; see TmaSmem)
    StepTablesS<P>* tsm = reinterpret_cast<StepTablesS<P>*>(base + SM::ring + SM::partials + SM::params);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + SM::ring + SM::partials + SM::params + SM::tables);
    // item table: entry s % kItems = (s << 32) | (ring offset in units << 8) | pieces for item s
    // (tile-major, 45 per tile), written with one 64-bit store
    // (producer p's block starts at bars + 3*kItems*p: full, empty, item table)
    volatile unsigned long long* items = reinterpret_cast<volatile unsigned long long*>(bars + 2 * kItems);
    const uint32_t tmem_full0 = smem_u32(bars + NPROD * 3 * kItems), tmem_empty0 = tmem_full0 + 64;
    int* start_of = reinterpret_cast<int*>(bars + NPROD * 3 * kItems + 16);  // ring offset per item in flight
    volatile int* abort_flag = start_of + NPROD * kItems;
    uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(start_of + NPROD * kItems) + 1;
    long long* woff = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(bars) + SM::bars_padded);
    float4* stage = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(bars) + SM::bars_padded + SM::woff);
    float2* scratch = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(bars) + SM::bars_padded + SM::woff +
                                                SM::stage);
    // Prandtl term: partial sums [quarter][component][x][lane] (20 rows), the centred third
    // moment [component][x][lane] (10 rows), then the per-velocity coefficients
    float* qreg = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(bars) + SM::bars_padded + SM::woff +
                                           SM::stage + SM::scratch);
    const uint32_t full0 = smem_u32(bars);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // tables into shared memory (sizeof is a multiple of 4)
        const int* src = reinterpret_cast<const int*>(&tpar);
        int* dstw = reinterpret_cast<int*>(tsm);
        for (int q = threadIdx.x; q < static_cast<int>(sizeof(StepTablesS<P>) / 4); q += blockDim.x) dstw[q] = src[q];
        if constexpr (PR) {
            float* pa = qreg + SM::kQRows * G::TX * 32;
            for (int q = threadIdx.x; q < kQ * 10; q += blockDim.x) pa[q] = prt.a[q / 10][q % 10];
        }
    }
    const StepTablesS<P>& t = *tsm;
    if (threadIdx.x == 0) {
        for (int e = 0; e < NPROD * 3 * kItems; ++e)
            if (e % (3 * kItems) < 2 * kItems) mbar_init(full0 + 8 * e, 1);  // full and empty
        for (int pp = 0; pp < NPROD; ++pp)
            for (int e = 0; e < kItems; ++e) items[pp * 3 * kItems + e] = ~0ull;
        for (int q = 0; q < 4; ++q)
            for (int b = 0; b < 2; ++b) {
                mbar_init(tmem_full0 + 8 * (q * 2 + b), q == 1 ? 2u : 3u);  // stream warps per quarter
                mbar_init(tmem_empty0 + 8 * (q * 2 + b), 1);
            }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // tensor memory for the streamed populations, freed by the same warp at the end
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_base_s)),
                     "r"(static_cast<uint32_t>(TC::alloc))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // the launch's tiles: a.cells[2] / CZ z-tiles starting at z-tile a.tz_begin, cells counted
    // from a.z0 (a slab's ghost cells lie below it; the source boxes of a slab's tiles stay in
    // its buffer, so they never wrap along z)
    const int ntx = a.cells[0] / CX, nty = (a.cells[1] + CY - 1) / CY, ntz = a.cells[2] / CZ;
    const int ntiles = ntx * nty * ntz;
    int* err_flag = a.flag_err;

    if (is_producer_warp(warp)) {
        // ------------------------------------------------ producer warps
        // Producer pp serves the velocities j = pp + NPROD*m (m < IPP), which are the pairs of
        // the stream warps c = pp (mod NPROD), through its own part of the box ring and its own
        // descriptors.  Per tile, lane m works out item m in parallel (box origin of the first
        // periodic image, image counts, shape, ring units).  Items then go out in order, in
        // batches: the releases of the oldest items in flight are confirmed together (one
        // lane per item), as many of the next items as fit are placed in the ring, and they
        // are announced and issued at once, one lane per item.  A producer that falls behind
        // thus issues larger batches instead of paying the mbarrier and TMA latencies once
        // per item.  The ring is reclaimed in item order.
        const int pp = producer_index(warp);
        const uint32_t pf0 = full0 + 8u * static_cast<uint32_t>(pp * 3 * kItems), pe0 = pf0 + 8u * kItems;
        volatile unsigned long long* pit = items + pp * 3 * kItems;
        int* pst = start_of + pp * kItems;
        long long* pwo = woff + pp * SM::woff_n;
        constexpr int RP = SM::ring_units / NPROD;  // ring units of this producer ...
        const int RB = pp * RP;                     // ... starting at this unit
        uint32_t s_tile = 0;  // number of the tile's first item
        uint32_t tail = 0;    // oldest item whose release is not confirmed yet
        int head = 0;         // ring unit where the next item goes (if it fits)
        uint32_t sent = 0;    // items issued
        bool ok = true;
        const uint32_t ring_u32 = smem_u32(ringb);
        const int cd[3] = {CX, CY, CZ};
        // the host-written abort request word, read one tile ahead so that its latency hides
        // behind a tile's work
        const volatile int* abort_req = reinterpret_cast<const volatile int*>(a.abort_req);
        int req_word = (lane == 0 && abort_req != nullptr) ? *abort_req : 0;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, s_tile += IPP) {
            // an abort request ends the launch at a tile boundary: the consumers leave through
            // the abort flag, this producer drains its copies (below)
            if (__shfl_sync(0xffffffffu, req_word, 0) != 0) {
                if (lane == 0) {
                    *abort_flag = 1;
                    if (err_flag != nullptr) atomicOr(err_flag, 4);
                }
                ok = false;
                break;
            }
            if (lane == 0 && abort_req != nullptr) req_word = *abort_req;
            int tc[3];
            tile_coords(tile, ntx, nty, ntz, tc);
            const int cb[3] = {tc[0] * CX * P, tc[1] * CY * P, ((tc[2] + a.tz_begin) * CZ + a.z0) * P};
            // meta: pieces m | nk_x << 4 | nk_y << 8 | nk_z << 12 | shape << 16 | cp.async << 20
            uint32_t meta[2];
            int crd[2][3];
            int units[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int mi = lane + 32 * h;
                const int j = pp + NPROD * mi;
                meta[h] = 0;
                units[h] = 0;
                crd[h][0] = crd[h][1] = crd[h][2] = 0;
                if (mi < IPP) {
                    int b0[3], klo[3], nk[3], sp[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        sp[d] = t.span[j][d];
                        b0[d] = cb[d] + t.kmin[j][d] * P;
                        const int need = (cd[d] + sp[d]) * P + 1;
                        klo[d] = floor_div(b0[d], a.N[d]);
                        nk[d] = floor_div(b0[d] + need - 1, a.N[d]) - klo[d] + 1;
                    }
                    const int npiece = nk[0] * nk[1] * nk[2];
                    const int shape = sp[0] + 2 * sp[1] + 4 * sp[2];
                    const bool tma_pieces = npiece <= kMaxPieces && npiece * G::piece_units(shape) <= RP;
                    const int m = tma_pieces ? npiece : 1;
                    units[h] = m * G::piece_units(shape);
                    const int x0 = b0[0] - (b0[0] & (G::AL - 1));  // 16-byte aligned pair index (floor)
                    crd[h][0] = XM * (x0 - klo[0] * a.N[0]);
                    crd[h][1] = b0[1] - klo[1] * a.N[1];
                    crd[h][2] = b0[2] - klo[2] * a.N[2];
                    meta[h] = static_cast<uint32_t>(m | (nk[0] << 4) | (nk[1] << 8) | (nk[2] << 12) | (shape << 16) |
                                                    ((tma_pieces ? 0 : 1) << 20));
                }
            }

            // per round of 32 items: inclusive prefix sums of the ring units over the lanes, and the
            // lanes whose item takes the cp.async path
            int incl_r[2] = {units[0], units[1]};
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = __shfl_up_sync(0xffffffffu, incl_r[h], o);
                    if (lane >= o) incl_r[h] += u;
                }
            }
            const uint32_t fbm_r[2] = {__ballot_sync(0xffffffffu, (meta[0] >> 20) & 1u),
                                       __ballot_sync(0xffffffffu, (meta[1] >> 20) & 1u)};

            int nxt = 0;  // first item of the tile not issued yet
            while (nxt < IPP) {
                const int h = nxt >> 5;
                const int lo = nxt & 31;
                const int nlane = h ? IPP - 32 : (IPP < 32 ? IPP : 32);  // items held in this round
                const uint32_t issued = s_tile + static_cast<uint32_t>(nxt);
                // confirm the releases of the oldest items in flight, in order
                int inflight = static_cast<int>(issued - tail);
                if (inflight > 0) {
                    const uint32_t x = tail + static_cast<uint32_t>(lane);
                    // (the oldest 8 at most: each lane's test is a separate shared-memory operation)
                    const bool rel = lane < inflight && lane < 8 && mbar_test_wait(pe0 + 8 * (x & KM), (x / kItems) & 1u);
                    const uint32_t rm = __ballot_sync(0xffffffffu, rel);
                    const int nrel = (~rm == 0u) ? 32 : __ffs(static_cast<int>(~rm)) - 1;
                    tail += static_cast<uint32_t>(nrel);
                    inflight -= nrel;
                }
                if (inflight == 0) head = 0;  // ring empty: start over at its beginning
                // Place the next items of this round: the longest run from the first one whose
                // ring units (the tile's prefix sums, taken from item lo on) fit in one free
                // region (the rest of the ring after `head`, or its start when that is too
                // short).  A cp.async item goes alone.
                const int tail_off = inflight > 0 ? pst[tail & KM] : 0;
                const int cap = min(nlane - lo, kItems - inflight);
                const uint32_t fbm = h ? fbm_r[1] : fbm_r[0];
                const bool first_fb = (fbm >> lo) & 1u;
                // candidates end before the first cp.async item after the first one
                const uint32_t fb_after = fbm & ~((2u << lo) - 1u);
                const int end = first_fb ? lo + 1 : (fb_after ? min(lo + cap, __ffs(static_cast<int>(fb_after)) - 1) : lo + cap);
                const int need_l = h ? units[1] : units[0];
                const int incl_l = h ? incl_r[1] : incl_r[0];
                const int excl_lo = __shfl_sync(0xffffffffu, incl_l - need_l, lo);
                const int first_need = __shfl_sync(0xffffffffu, need_l, lo);
                const int incl = incl_l - excl_lo;  // units of items lo .. lane
                int base = -1, limit = 0;
                if (inflight == 0) {
                    base = head;
                    limit = RP;
                } else if (head > tail_off) {
                    if (head + first_need <= RP) {
                        base = head;
                        limit = RP;
                    } else if (first_need <= tail_off) {
                        base = 0;
                        limit = tail_off;
                    }
                } else if (head < tail_off) {
                    base = head;
                    limit = tail_off;
                }
                const bool fits = base >= 0 && lane >= lo && lane < end && base + incl <= limit;
                const uint32_t fm = __ballot_sync(0xffffffffu, fits) >> lo;
                const int nb = (~fm == 0u) ? 32 - lo : __ffs(static_cast<int>(~fm)) - 1;
                const int my_off = base + incl - need_l;
                if (nb > 0) head = base + __shfl_sync(0xffffffffu, incl, lo + nb - 1);
                if (nb == 0) {
                    // nothing fits: wait (blocking, bounded) for the oldest item's release
                    int stop = 0;
                    if (lane == 0 && !mbar_wait_bounded(pe0 + 8 * (tail & KM), (tail / kItems) & 1u, abort_flag,
                                                        err_flag, a.wait_ns))
                        stop = 1;
                    if (__shfl_sync(0xffffffffu, stop, 0)) {
                        ok = false;
                        break;
                    }
                    ++tail;
                    continue;
                }
                // announce and issue the batch, one lane per item
                const bool mine = lane >= lo && lane < lo + nb;
                if (mine) {
                    const uint32_t s = issued + static_cast<uint32_t>(lane - lo);
                    const uint32_t mt = h ? meta[1] : meta[0];
                    const int m = static_cast<int>(mt & 15u);
                    const uint32_t e = s & KM;
                    pst[e] = my_off;
                    pit[e] = (static_cast<unsigned long long>(s) << 32) | (static_cast<uint32_t>(RB + my_off) << 8) |
                               static_cast<uint32_t>(m);
                    if (!first_fb) {
                        const int shape = static_cast<int>((mt >> 16) & 7u);
                        const CUtensorMap* map = &maps.m[shape];
                        const uint32_t bytes = static_cast<uint32_t>(G::box_bytes(shape));
                        const uint32_t pstride = static_cast<uint32_t>(G::piece_units(shape)) * 128u;
                        const int nkx = static_cast<int>((mt >> 4) & 15u), nky = static_cast<int>((mt >> 8) & 15u),
                                  nkz = static_cast<int>((mt >> 12) & 15u);
                        const int cx = h ? crd[1][0] : crd[0][0], cy = h ? crd[1][1] : crd[0][1],
                                  cz = h ? crd[1][2] : crd[0][2];
                        const int j = pp + NPROD * (lane + 32 * h);
                        const uint32_t full = pf0 + 8 * e;
                        mbar_arrive_expect_tx(full, bytes * static_cast<uint32_t>(m));
                        uint32_t dst = ring_u32 + static_cast<uint32_t>(RB + my_off) * 128u;
                        for (int qz = 0; qz < nkz; ++qz)
                            for (int qy = 0; qy < nky; ++qy)
                                for (int qx = 0; qx < nkx; ++qx, dst += pstride)
                                    tma_load_4d(dst, map, cx - XM * qx * a.N[0], cy - qy * a.N[1], cz - qz * a.N[2], j,
                                                full);
                    }
                }
                if (first_fb) {
                    const int j = pp + NPROD * nxt;
                    const uint32_t e = issued & KM;
                    const int foff = __shfl_sync(0xffffffffu, my_off, lo);
                    int b0[3], sp[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        sp[d] = t.span[j][d];
                        b0[d] = cb[d] + t.kmin[j][d] * P;
                    }
                    const int x0 = b0[0] - (b0[0] & (G::AL - 1));
                    const uint32_t dst = ring_u32 + static_cast<uint32_t>(RB + foff) * 128u;
                    const uint32_t full = pf0 + 8 * e;
                    // the box overlaps more periodic images than there are pieces: 16-byte copies
                    // from the wrapped positions, in the layout of the box's shape.  A chunk is
                    // AL (f,g) pairs at an x that is a multiple of AL and N[0] is a multiple of AL,
                    // so a chunk never straddles the boundary.  The wrapped offsets (in stored
                    // elements) of the box's planes, rows and chunks are computed once per box
                    // into a table.
                    const S* src = static_cast<const S*>(a.src) + 2LL * j * a.nn;
                    const int XP = G::xpairs_s(sp[0]), YR = G::rows(sp[1]), ZP = G::planes(sp[2]);
                    const int CH = XP / G::AL;
                    const int nchunk = ZP * YR * CH;
                    if (lane < ZP) pwo[lane] = 2LL * wrapi(b0[2] + lane, a.N[2]) * a.N[1] * a.N[0];
                    if (lane < YR) pwo[G::BZ + lane] = 2LL * wrapi(b0[1] + lane, a.N[1]) * a.N[0];
                    if (lane < CH) pwo[G::BZ + G::BY + lane] = 2LL * wrapi(x0 + G::AL * lane, a.N[0]);
                    __syncwarp();
                    for (int q = lane; q < nchunk; q += 32) {
                        const int row = q / CH;
                        const int c = q - row * CH;
                        const int z = row / YR, y = row - z * YR;
                        const long long off = pwo[z] + pwo[G::BZ + y] + pwo[G::BZ + G::BY + c];
                        cp_async16(dst + static_cast<uint32_t>((row * XP + G::AL * c) * G::PB), src + off);
                    }
                    __syncwarp();  // the table is rewritten for the next such box
                    cp_async_mbar_arrive(full);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full);
                }
                __syncwarp();  // ring offsets written by the issuing lanes are read by all
                nxt += nb;
                sent = issued + static_cast<uint32_t>(nb);
            }
        }
        // Drain, on every exit: wait (bounded, whatever the abort flag says) until the fills
        // of every item whose release is not confirmed have landed, so that the CTA never
        // ends with a bulk-tensor or cp.async copy still writing its shared memory.  This
        // matters when the consumers left early (abort) while this producer went on and
        // issued its last items: those items have no consumer that waits for them.  In a
        // normal run every such item was consumed, its fill phase has completed and each
        // test passes at once.  The items tail .. sent-1 are the last uses of their
        // descriptors (at most kItems of them), so one parity bit tells their phases apart.
        // A fill lands in bounded time (a TMA or cp.async read of global memory); the 2 s
        // limit is only reached if an item's byte count disagreed with its copies, in which
        // case nothing is left in flight either.
        {
            volatile int keep_waiting = 0;
            for (uint32_t x = tail; x != sent; ++x)
                mbar_wait_bounded(pf0 + 8 * (x & KM), (x / kItems) & 1u, &keep_waiting, nullptr, kWaitNs);
        }
        return;
    }


    // ---------------------------------------------------- stream warps
    // Stream warp c streams its pairs pair_of(c, k) of every tile of the CTA into tensor-memory
    // buffer it & 1 of its lane quarter (its warp index mod 4), then hands the buffer to the
    // quarter's epilogue warp (tmem_full); before reusing a buffer it waits until that warp has
    // read it (tmem_empty).
    const int ncta = ntiles > static_cast<int>(blockIdx.x)
                         ? (ntiles - 1 - static_cast<int>(blockIdx.x)) / static_cast<int>(gridDim.x) + 1
                         : 0;
    const int oz_l = lane / G::TY, oy_l = lane % G::TY;
    if (is_stream_warp(warp)) {
        const int c = stream_index(warp), qd = warp & 3, npw = pairs_of(c);
        const uint32_t pbase = static_cast<uint32_t>((c % NPROD) * 3 * kItems);  // its producer's block
        const bool row_lane = lane < G::ROWS;
        const uint32_t tmem_warp = *tmem_base_s + (static_cast<uint32_t>(qd * 32) << 16) +
                                   static_cast<uint32_t>((warp >> 2) * TC::per_warp);
        for (int it = 0; it < ncta; ++it) {
            if (*abort_flag) break;
            const int bf = it & 1;
            const int tile = static_cast<int>(blockIdx.x) + it * static_cast<int>(gridDim.x);
            int tc[3];
            tile_coords(tile, ntx, nty, ntz, tc);
            const int c0[3] = {tc[0] * CX, tc[1] * CY, (tc[2] + a.tz_begin) * CZ + a.z0};
            if (it >= 2)
                mbar_wait_bounded(tmem_empty0 + 8 * (qd * 2 + bf), static_cast<uint32_t>((it - 2) >> 1) & 1u, abort_flag,
                                  err_flag, a.wait_ns);
            tc_fence_after();
            const uint32_t tbuf = tmem_warp + static_cast<uint32_t>(bf * TC::per_buf);
#pragma unroll 1
            for (int k = 0; k < npw; ++k) {
                const int j = pair_of(c, k);
                const uint32_t s = static_cast<uint32_t>(it) * IPP + static_cast<uint32_t>(j / NPROD);
                // Where the item sits in the ring.  The producer announces item s only once item
                // s - kItems has released the same descriptor, so its full barrier is then at most
                // one phase ahead of the phase awaited below (one parity bit cannot tell more apart).
                const uint32_t e = s & KM;
                const uint32_t word = wait_item_bounded(items + pbase + e, s, abort_flag, err_flag, a.wait_ns);
                const int m = static_cast<int>(word & 15u);  // (0 only when the wait gave up)
                // Whether this item's copies have landed.  An item whose wait gave up (abort)
                // is not released below: its fill may still be writing the box, and an
                // unreleased item stays in the producer's drain.
                const bool filled =
                    m > 0 && mbar_wait_bounded(full0 + 8 * (pbase + e), (s / kItems) & 1u, abort_flag, err_flag, a.wait_ns);
                const unsigned char* sbox = ringb + static_cast<size_t>(word >> 8) * 128;
                // the first used pair of a box row: ox0s in the stored row (which starts at a
                // multiple of AL), ox0 = 0 or 1 in the FP32 row the passes use, which starts
                // xs stored pairs into the stored row (xs = 0 for FP32 storage: the same row)
                const int ox0s = ((c0[0] + t.kmin[j][0]) * P) & (G::AL - 1);
                const int ox0 = ox0s & 1, xs = ox0s - ox0;
                // the box's shape: FP32 rows of XP pairs, planes of PL pairs; stored rows of XPS
                // pairs, planes of PLS pairs; pieces PSTRIDE bytes apart
                const int sx = t.span[j][0], sy = t.span[j][1], sz = t.span[j][2];
                const int XP = G::xpairs(sx), PL = G::rows(sy) * XP;
                const int XPS = G::xpairs_s(sx), PLS = G::rows(sy) * XPS;
                const int PSTRIDE = G::piece_units(sx + 2 * sy + 4 * sz) * 128;
                // where the passes run: in place in the ring (FP32), in the warp's scratch (16-bit)
                float2* box = G::kF32 ? reinterpret_cast<float2*>(const_cast<unsigned char*>(sbox))
                                      : scratch + static_cast<size_t>(c) * G::SCRATCH_F2;

                // z pass: column (y, xb) of the box, NZ planes -> output planes 0..TZ-1 of the
                // FP32 box (in place for FP32 storage; 16-bit pairs are widened on the way)
                auto z_pass = [&](auto nz) {
                    constexpr int NZ = decltype(nz)::value;
                    float2 wz[P][P + 1];
                    bool kz[P];
#pragma unroll
                    for (int az = 0; az < P; ++az) {
                        kz[az] = t.kc[j][2][az] != 0;
#pragma unroll
                        for (int l = 0; l <= P; ++l) wz[az][l] = make_float2(t.lw[j][2][az][l], t.lw[j][2][az][l]);
                    }
                    // two adjacent columns per lane: 16-byte loads and stores of FP32 pairs (PL is
                    // even and the box starts on a 128-byte boundary), 8-byte loads of 16-bit pairs
                    // (even pair index: xs, XPS and the column are even)
                    const int nq = PL >> 1, XQ = XP >> 1;
                    float4* box4 = reinterpret_cast<float4*>(box);
#pragma unroll 1
                    for (int e2 = lane; e2 < nq; e2 += 32) {
                        float2 va[NZ], vb[NZ];
                        int srow = 0;  // 16-bit: the column pair's index in a stored plane, in 8-byte units
                        if constexpr (!G::kF32) {
                            const int y = e2 / XQ;
                            srow = ((y * XPS + xs) >> 1) + (e2 - y * XQ);
                        } else {
                            (void)srow;
                            (void)XQ;
                        }
                        if constexpr (G::kF32) {
                            const float4* b0 = reinterpret_cast<const float4*>(sbox);
#pragma unroll
                            for (int z = 0; z < NZ; ++z) {
                                const float4 q4 = b0[z * nq + e2];
                                va[z] = make_float2(q4.x, q4.y);
                                vb[z] = make_float2(q4.z, q4.w);
                            }
                        } else {
                            const uint2* b0 = reinterpret_cast<const uint2*>(sbox);
#pragma unroll
                            for (int z = 0; z < NZ; ++z) {
                                const uint2 u = b0[z * (PLS >> 1) + srow];
                                va[z] = widen_pair<S>(u.x);
                                vb[z] = widen_pair<S>(u.y);
                            }
                        }
                        // the other periodic images of a box that crosses the boundary (each is
                        // zero outside the domain, so their sum is the wrapped box)
                        for (int q = 1; q < m; ++q) {
                            if constexpr (G::kF32) {
                                const float4* bq = reinterpret_cast<const float4*>(sbox + q * PSTRIDE);
#pragma unroll
                                for (int z = 0; z < NZ; ++z) {
                                    const float4 u = bq[z * nq + e2];
                                    va[z].x += u.x;
                                    va[z].y += u.y;
                                    vb[z].x += u.z;
                                    vb[z].y += u.w;
                                }
                            } else {
                                const uint2* bq = reinterpret_cast<const uint2*>(sbox + q * PSTRIDE);
#pragma unroll
                                for (int z = 0; z < NZ; ++z) {
                                    const uint2 u = bq[z * (PLS >> 1) + srow];
                                    const float2 ua = widen_pair<S>(u.x), ub = widen_pair<S>(u.y);
                                    va[z].x += ua.x;
                                    va[z].y += ua.y;
                                    vb[z].x += ub.x;
                                    vb[z].y += ub.y;
                                }
                            }
                        }
#pragma unroll
                        for (int oz = 0; oz < G::TZ; ++oz) {
                            const int cz = oz / P, az = oz % P;
                            float2 oa = make_float2(0.f, 0.f), ob = make_float2(0.f, 0.f);
                            if constexpr (NZ == G::BZ) {
                                if (kz[az]) {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) {
                                        oa = ffma2(va[(cz + 1) * P + l], wz[az][l], oa);
                                        ob = ffma2(vb[(cz + 1) * P + l], wz[az][l], ob);
                                    }
                                } else {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) {
                                        oa = ffma2(va[cz * P + l], wz[az][l], oa);
                                        ob = ffma2(vb[cz * P + l], wz[az][l], ob);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int l = 0; l <= P; ++l) {
                                    oa = ffma2(va[cz * P + l], wz[az][l], oa);
                                    ob = ffma2(vb[cz * P + l], wz[az][l], ob);
                                }
                            }
                            box4[oz * nq + e2] = make_float4(oa.x, oa.y, ob.x, ob.y);
                        }
                    }
                };
                if (sz)
                    z_pass(IntC<G::BZ>{});
                else
                    z_pass(IntC<G::BZ0>{});
                __syncwarp();
                if constexpr (!G::kF32) {
                    // the stored box has been read (into the scratch): release it now
                    if (lane == 0 && filled) mbar_arrive(full0 + 8 * (pbase + kItems + e));
                }
                // y pass, in place: column (oz, xb), NY rows -> output rows 0..TY-1
                auto y_pass = [&](auto ny) {
                    constexpr int NY = decltype(ny)::value;
                    float2 wy[P][P + 1];
                    bool ky[P];
#pragma unroll
                    for (int ay = 0; ay < P; ++ay) {
                        ky[ay] = t.kc[j][1][ay] != 0;
#pragma unroll
                        for (int l = 0; l <= P; ++l) wy[ay][l] = make_float2(t.lw[j][1][ay][l], t.lw[j][1][ay][l]);
                    }
                    // two adjacent columns per lane: 16-byte loads and stores (XP is even).  A
                    // full-height box (NY == BY) has planes of an odd number of 16-byte columns,
                    // so consecutive lanes over (oz, xq) would put two planes' columns in one
                    // eighth of the warp on the same banks; there lane 8 oz + xq takes column
                    // (oz, xq), each eighth reading within one plane (conflict free).
                    const int XQ = XP >> 1;
                    float4* box4 = reinterpret_cast<float4*>(box);
                    constexpr bool kByPlane = NY == G::BY && G::TZ <= 4 && G::BXP / 2 <= 8;
                    const int ncol = kByPlane ? 32 : G::TZ * XQ;
#pragma unroll 1
                    for (int e = lane; e < ncol; e += 32) {
                        const int oz = kByPlane ? e >> 3 : e / XQ, xq = kByPlane ? e & 7 : e - oz * XQ;
                        if (kByPlane && (oz >= G::TZ || xq >= XQ)) continue;
                        float4* col = box4 + oz * (PL >> 1) + xq;
                        float2 va[NY], vb[NY];
#pragma unroll
                        for (int y = 0; y < NY; ++y) {
                            const float4 q4 = col[y * XQ];
                            va[y] = make_float2(q4.x, q4.y);
                            vb[y] = make_float2(q4.z, q4.w);
                        }
#pragma unroll
                        for (int oy = 0; oy < G::TY; ++oy) {
                            const int cy = oy / P, ay = oy % P;
                            float2 oa = make_float2(0.f, 0.f), ob = make_float2(0.f, 0.f);
                            if constexpr (NY == G::BY) {
                                if (ky[ay]) {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) {
                                        oa = ffma2(va[(cy + 1) * P + l], wy[ay][l], oa);
                                        ob = ffma2(vb[(cy + 1) * P + l], wy[ay][l], ob);
                                    }
                                } else {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) {
                                        oa = ffma2(va[cy * P + l], wy[ay][l], oa);
                                        ob = ffma2(vb[cy * P + l], wy[ay][l], ob);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int l = 0; l <= P; ++l) {
                                    oa = ffma2(va[cy * P + l], wy[ay][l], oa);
                                    ob = ffma2(vb[cy * P + l], wy[ay][l], ob);
                                }
                            }
                            col[oy * XQ] = make_float4(oa.x, oa.y, ob.x, ob.y);
                        }
                    }
                };
                if (sy)
                    y_pass(IntC<G::BY>{});
                else
                    y_pass(IntC<G::BY0>{});
                __syncwarp();
                // x pass: lane = x-row (oz, oy) of the tile, NX pairs from the row's start
                float res[2 * G::TX];
                auto x_pass = [&](auto nx) {
                    constexpr int NX = decltype(nx)::value;
                    float2 wx[P][P + 1];
                    bool kx[P];
#pragma unroll
                    for (int ax = 0; ax < P; ++ax) {
                        kx[ax] = t.kc[j][0][ax] != 0;
#pragma unroll
                        for (int l = 0; l <= P; ++l) wx[ax][l] = make_float2(t.lw[j][0][ax][l], t.lw[j][0][ax][l]);
                    }
                    // the row from its even start in 16-byte loads (rows start on an even pair;
                    // these are free of bank conflicts where 8-byte loads of the odd-stride rows
                    // are not), the first pair used being ox0 = 0 or 1
                    constexpr int K = (NX + 2) / 2;
                    static_assert(2 * K <= (NX == G::BX ? G::BXP : G::BXP0), "row loads stay in the row");
                    float2 u[2 * K];
                    const float4* row4 = reinterpret_cast<const float4*>(box + oz_l * PL + oy_l * XP);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        const float4 q4 = row_lane ? row4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                        u[2 * q] = make_float2(q4.x, q4.y);
                        u[2 * q + 1] = make_float2(q4.z, q4.w);
                    }
                    auto interp = [&](auto off) {
                        constexpr int O = decltype(off)::value;
#pragma unroll
                        for (int ox = 0; ox < G::TX; ++ox) {
                            const int cx = ox / P, ax = ox % P;
                            float2 o = make_float2(0.f, 0.f);
                            if constexpr (NX == G::BX) {
                                if (kx[ax]) {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) o = ffma2(u[O + (cx + 1) * P + l], wx[ax][l], o);
                                } else {
#pragma unroll
                                    for (int l = 0; l <= P; ++l) o = ffma2(u[O + cx * P + l], wx[ax][l], o);
                                }
                            } else {
#pragma unroll
                                for (int l = 0; l <= P; ++l) o = ffma2(u[O + cx * P + l], wx[ax][l], o);
                            }
                            res[2 * ox] = o.x;
                            res[2 * ox + 1] = o.y;
                        }
                    };
                    if (ox0)
                        interp(IntC<1>{});
                    else
                        interp(IntC<0>{});
                };
                if (sx)
                    x_pass(IntC<G::BX>{});
                else
                    x_pass(IntC<G::BX0>{});
                if constexpr (G::kF32) {
                    // the slot was written in place (generic proxy); order that before the next
                    // TMA fill
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0 && filled) mbar_arrive(full0 + 8 * (pbase + kItems + e));
                } else {
                    __syncwarp();  // the scratch is rewritten by the next pair's z pass
                }

                // park the pair in tensor memory
                tmem_store_row<G::TX>(tbuf + static_cast<uint32_t>(k * G::PCS), res);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_full0 + 8 * (qd * 2 + bf));
        }
    }
    // ---------------------------------------------------- epilogue warps
    // One per lane quarter.  Per tile: the moment sums of the quarter's pairs (streamed by
    // warps q, q + 4, q + 8; q + 4, q + 8 in quarter 1), the sum over the quarters in a fixed
    // order and the per-node parameters (each epilogue warp a share of the nodes), then the BGK
    // collision and the stores of the quarter's pairs.  The epilogue warps meet at named
    // barrier 2.
    else if (is_epilogue_warp(warp)) {
        const int ep = epilogue_index(warp);  // 0 .. NE-1: share of the nodes whose parameters it forms
        const int qd = warp & 3;              // the lane quarter it reads (= ep)
        constexpr int nsw = 3;                // stream warp slots in the quarter: warps qd, qd + 4, qd + 8
        const int sw0 = qd == 1 ? 1 : 0;      // (warp 1 is the producer)
        const uint32_t tq = *tmem_base_s + (static_cast<uint32_t>(qd * 32) << 16);
        constexpr int QS = G::TX * 32;  // stride between parameters
        constexpr int XS = (G::TX + NE - 1) / NE;  // node columns per epilogue warp (the last one fewer)
        for (int it = 0; it < ncta; ++it) {
            if (epilogue_barrier_or(*abort_flag)) break;
            const int bf = it & 1;
            const int tile = static_cast<int>(blockIdx.x) + it * static_cast<int>(gridDim.x);
            int tc[3];
            tile_coords(tile, ntx, nty, ntz, tc);
            const int c0[3] = {tc[0] * CX, tc[1] * CY, (tc[2] + a.tz_begin) * CZ + a.z0};
            const uint32_t tb = tq + static_cast<uint32_t>(bf * TC::per_buf);
            mbar_wait_bounded(tmem_full0 + 8 * (qd * 2 + bf), static_cast<uint32_t>(it >> 1) & 1u, abort_flag, err_flag,
                              a.wait_ns);
            tc_fence_after();
            // moment contributions of the quarter's pairs (rho, m_x, m_y, m_z, 2 rho E; Eq. moments)
            if constexpr (KC) {
                // compensated: a running sum and its exact rounding errors per moment and node,
                // CH node columns at a time (8-node rows in two halves: measured faster than
                // whole rows there, 1.05 against 1.12 ms per 128^3 step; 6-node rows whole);
                // the sums go to rows [quarter][moment], the error terms to the 20 rows after them
                constexpr int CH = G::TX == 8 ? 4 : G::TX;
                float* pc = part + static_cast<size_t>(qd) * 5 * QS + lane;
                float* pe = pc + 20 * QS;
#pragma unroll 1
                for (int x0 = 0; x0 < G::TX; x0 += CH) {
                    CompSum<float> cs[5][CH];
                    for (int sw = sw0; sw < nsw; ++sw) {
                        const int cw = stream_index(qd + 4 * sw), npw = pairs_of(cw);
#pragma unroll 1
                        for (int k = 0; k < npw; ++k) {
                            const int j = pair_of(cw, k);
                            float v[2 * CH];
                            tmem_load_nodes<CH>(
                                tb + static_cast<uint32_t>(sw * TC::per_warp + k * G::PCS + 2 * x0), v);
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            const float xix = t.xi[j][0], xiy = t.xi[j][1], xiz = t.xi[j][2];
                            const float x2 = static_cast<float>(shell_xi2(shell_of(j)));
                            if constexpr (G::kF32) {
#pragma unroll
                                for (int x = 0; x < CH; ++x) {
                                    const float f = v[2 * x], g = v[2 * x + 1];
                                    cs[0][x].add(f);
                                    cs[1][x].add_prod(f, xix);
                                    cs[2][x].add_prod(f, xiy);
                                    cs[3][x].add_prod(f, xiz);
                                    cs[4][x].add_prod(f, x2);
                                    cs[4][x].add(g);
                                }
                            } else {
                                const float wj = t.w[j];
                                const float wx = wj * xix, wy = wj * xiy, wz = wj * xiz, wx2 = wj * x2;
#pragma unroll
                                for (int x = 0; x < CH; ++x) {
                                    const float d = v[2 * x], dg = v[2 * x + 1];
                                    cs[0][x].add_prod(wj, d);
                                    cs[1][x].add_prod(wx, d);
                                    cs[2][x].add_prod(wy, d);
                                    cs[3][x].add_prod(wz, d);
                                    cs[4][x].add_prod(wx2, d);
                                    cs[4][x].add_prod(wj, dg);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 5; ++q)
#pragma unroll
                        for (int x = 0; x < CH; ++x) {
                            pc[q * QS + (x0 + x) * 32] = cs[q][x].s;
                            pe[q * QS + (x0 + x) * 32] = cs[q][x].c;
                        }
                }
            } else {
                float pm[5][G::TX];
#pragma unroll
                for (int q = 0; q < 5; ++q)
#pragma unroll
                    for (int x = 0; x < G::TX; ++x) pm[q][x] = 0.f;
                for (int sw = sw0; sw < nsw; ++sw) {
                    const int cw = stream_index(qd + 4 * sw), npw = pairs_of(cw);
#pragma unroll 1
                    for (int k = 0; k < npw; ++k) {
                        const int j = pair_of(cw, k);
                        float v[2 * G::TX];
                        tmem_load_row<G::TX>(tb + static_cast<uint32_t>(sw * TC::per_warp + k * G::PCS), v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        const float xix = t.xi[j][0], xiy = t.xi[j][1], xiz = t.xi[j][2];
                        const float x2 = static_cast<float>(shell_xi2(shell_of(j)));
                        if constexpr (G::kF32) {
#pragma unroll
                            for (int x = 0; x < G::TX; ++x) {
                                const float f = v[2 * x], g = v[2 * x + 1];
                                pm[0][x] += f;
                                pm[1][x] += f * xix;
                                pm[2][x] += f * xiy;
                                pm[3][x] += f * xiz;
                                pm[4][x] += f * x2 + g;
                            }
                        } else {
                            // deviation sums: rho - rho0, rho u and sum w (|xi|^2 d + d_g)
                            const float wj = t.w[j];
#pragma unroll
                            for (int x = 0; x < G::TX; ++x) {
                                const float wd = wj * v[2 * x], g = v[2 * x + 1];
                                pm[0][x] += wd;
                                pm[1][x] += wd * xix;
                                pm[2][x] += wd * xiy;
                                pm[3][x] += wd * xiz;
                                pm[4][x] += wd * x2 + wj * g;
                            }
                        }
                    }
                }
                // layout [quarter][moment][x][lane] (node = lane*TX + x): contiguous lane accesses
                float* pc = part + static_cast<size_t>(qd) * 5 * QS + lane;
#pragma unroll
                for (int q = 0; q < 5; ++q)
#pragma unroll
                    for (int x = 0; x < G::TX; ++x) pc[q * QS + x * 32] = pm[q][x];
            }
            epilogue_barrier_or(0);
            // per-node moments (quarters summed in a fixed order), tau, equilibrium coefficients
            // (Eq. discreteEquilibrium, Sutherland's law) of this warp's share of the nodes.  A
            // lane's row exists if it is one of the tile's x-rows and, in a partial tile, inside
            // the mesh; rows that do not exist are neither checked nor stored.
            const bool row_ok =
                (G::ROWS == 32 || lane < G::ROWS) && (!kRaggedY || c0[1] * P + oy_l < a.cells[1] * P);
#pragma unroll
            for (int xx = 0; xx < XS; ++xx) {
                const int x = ep * XS + xx;
                if (x >= G::TX) break;
                float m[5];
                [[maybe_unused]] CompSum<float> cm[5];  // compensated sums: the quarters' partials
                if constexpr (KC) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq)
                            cm[q].add_partial(part[(qq * 5 + q) * QS + x * 32 + lane],
                                              part[(20 + qq * 5 + q) * QS + x * 32 + lane]);
                        m[q] = cm[q].value();
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        m[q] = ((part[(0 * 5 + q) * QS + x * 32 + lane] + part[(1 * 5 + q) * QS + x * 32 + lane]) +
                                part[(2 * 5 + q) * QS + x * 32 + lane]) +
                               part[(3 * 5 + q) * QS + x * 32 + lane];
                }
                float* pn = prm + x * 32 + lane;
                if constexpr (G::kF32) {
                    const float rho = m[0];
                    const float inv_rho = 1.0f / rho;
                    const float ux = m[1] * inv_rho, uy = m[2] * inv_rho, uz = m[3] * inv_rho;
                    const float usq = ux * ux + uy * uy + uz * uz;
                    float T;
                    if constexpr (KC) {
                        // 2 rho E - rho |u|^2 = 2 rho E - m . u, compensated
                        CompSum<float> e = cm[4];
                        e.add_prod(-m[1], ux);
                        e.add_prod(-m[2], uy);
                        e.add_prod(-m[3], uz);
                        T = e.value() * inv_rho * static_cast<float>(a.inv_2cv);
                    } else {
                        T = (m[4] * inv_rho - usq) * static_cast<float>(a.inv_2cv);
                    }
                    if (a.flag != nullptr && row_ok && !(rho > 0.f && T > 0.f && isfinite(rho) && isfinite(T)))
                        atomicOr(a.flag, 1);
                    const float tau_r = static_cast<float>(a.mu_over_dt) * sutherland(T) / (rho * T) + 0.5f;
                    const EqCoef<float> ec = eq_coefficients(usq, T - 1.0f);
                    pn[0 * QS] = rho;
                    pn[1 * QS] = ux;
                    pn[2 * QS] = uy;
                    pn[3 * QS] = uz;
                    pn[4 * QS] = static_cast<float>(a.gfac) * T;
                    pn[5 * QS] = 1.0f / tau_r;
                    if constexpr (PR) {
                        // App. D: the term relaxes with tau_Pr = (tau - 1/2) / Pr + 1/2
                        const float tau_pr = (tau_r - 0.5f) * static_cast<float>(a.inv_pr) + 0.5f;
                        pn[18 * QS] = 1.0f / tau_r - 1.0f / tau_pr;
                    }
#pragma unroll
                    for (int sh = 0; sh < 4; ++sh) {
                        pn[(6 + sh) * QS] = ec.c0[sh];
                        pn[(10 + sh) * QS] = ec.c1[sh];
                        pn[(14 + sh) * QS] = ec.c2[sh];
                    }
                } else {
                    // from the deviation sums with the quadrature identities sum w = 1,
                    // sum w xi = 0, sum w |xi|^2 = D (the generic kernel's deviation collision):
                    // 2 C_v rho (T - T0) = sum w (|xi|^2 d + d_g) + D rho0 (1 - T0) - rho |u|^2
                    //                      - 2 C_v T0 (rho - rho0)
                    const float rho0 = static_cast<float>(a.rho0), T0 = static_cast<float>(a.T0);
                    const float two_cv = static_cast<float>(1.0 / a.inv_2cv), gfac = static_cast<float>(a.gfac);
                    const float drho = m[0];
                    const float rho = rho0 + drho;
                    const float inv_rho = 1.0f / rho;
                    const float ux = m[1] * inv_rho, uy = m[2] * inv_rho, uz = m[3] * inv_rho;
                    const float usq = ux * ux + uy * uy + uz * uz;
                    float dT;
                    if constexpr (KC) {
                        // every term of the balance compensated, rho |u|^2 as m . u
                        CompSum<float> e = cm[4];
                        e.add(3.0f * rho0 * (1.0f - T0));
                        e.add_prod(-m[1], ux);
                        e.add_prod(-m[2], uy);
                        e.add_prod(-m[3], uz);
                        e.add_prod(-two_cv * T0, drho);
                        dT = e.value() * inv_rho / two_cv;
                    } else {
                        dT = (m[4] + 3.0f * rho0 * (1.0f - T0) - rho * usq - two_cv * T0 * drho) * inv_rho / two_cv;
                    }
                    const float T = T0 + dT;
                    if (a.flag != nullptr && row_ok && !(rho > 0.f && T > 0.f && isfinite(rho) && isfinite(T)))
                        atomicOr(a.flag, 1);
                    const float tau_r = static_cast<float>(a.mu_over_dt) * sutherland(T) / (rho * T) + 0.5f;
                    const EqCoef<float> ec = eq_coefficients(usq, T - 1.0f);
                    const float th = T - 1.0f;
                    pn[0 * QS] = rho;
                    pn[1 * QS] = ux;
                    pn[2 * QS] = uy;
                    pn[3 * QS] = uz;
                    pn[4 * QS] = 1.0f / tau_r;
                    pn[5 * QS] = drho;
                    pn[6 * QS] = gfac * T * rho;
                    pn[7 * QS] = gfac * (dT * rho + T0 * drho);
#pragma unroll
                    for (int sh = 0; sh < 4; ++sh) {
                        // c0 - 1 without forming c0 (which is 1 + O(u^2, th))
                        const float x2 = static_cast<float>(shell_xi2(sh));
                        pn[(8 + sh) * QS] = -0.5f * usq + 0.5f * th * (x2 - 3.0f) + 0.125f * usq * usq +
                                            0.25f * th * usq * (5.0f - x2) +
                                            0.125f * th * th * (x2 * x2 - 10.0f * x2 + 15.0f);
                        pn[(12 + sh) * QS] = ec.c1[sh];
                        pn[(16 + sh) * QS] = ec.c2[sh];
                    }
                }
            }
            epilogue_barrier_or(0);
            float* qall = qreg + 20 * QS;  // Prandtl term: Qbar per node, 10 rows
            if constexpr (PR) {
                // App. D: centred third moment Qbar_abc = sum_i f_i c_a c_b c_c (c = xi_i - u)
                // of the streamed f at each node, from the quarter's pairs (a second pass over
                // its tensor-memory buffer) in two rounds of five components and two halves
                // of the lane's nodes (registers), the quarters' partial sums summed through
                // shared memory in a fixed order, as the moments are
                constexpr int NH = G::TX / 2;
                float* qpart = qreg;
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        float acc[5][NH], uxh[NH], uyh[NH], uzh[NH];
#pragma unroll
                        for (int n = 0; n < NH; ++n) {
                            const float* pn = prm + (hh * NH + n) * 32 + lane;
                            uxh[n] = pn[1 * QS];
                            uyh[n] = pn[2 * QS];
                            uzh[n] = pn[3 * QS];
#pragma unroll
                            for (int c = 0; c < 5; ++c) acc[c][n] = 0.f;
                        }
                        for (int sw = sw0; sw < nsw; ++sw) {
                            const int cw = stream_index(qd + 4 * sw), npw = pairs_of(cw);
#pragma unroll 1
                            for (int k = 0; k < npw; ++k) {
                                const int j = pair_of(cw, k);
                                float v[2 * G::TX];
                                tmem_load_row<G::TX>(tb + static_cast<uint32_t>(sw * TC::per_warp + k * G::PCS), v);
                                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                                const float xix = t.xi[j][0], xiy = t.xi[j][1], xiz = t.xi[j][2];
#pragma unroll
                                for (int n = 0; n < NH; ++n) {
                                    const float f = v[2 * (hh * NH + n)];
                                    const float cx = xix - uxh[n], cy = xiy - uyh[n], cz = xiz - uzh[n];
                                    const float fx = f * cx, fy = f * cy, fz = f * cz;
                                    if (r == 0) {
                                        acc[0][n] += fx * cx * cx;  // xxx
                                        acc[1][n] += fy * cy * cy;  // yyy
                                        acc[2][n] += fz * cz * cz;  // zzz
                                        acc[3][n] += fx * cx * cy;  // xxy
                                        acc[4][n] += fx * cx * cz;  // xxz
                                    } else {
                                        acc[0][n] += fy * cy * cx;  // yyx
                                        acc[1][n] += fy * cy * cz;  // yyz
                                        acc[2][n] += fz * cz * cx;  // zzx
                                        acc[3][n] += fz * cz * cy;  // zzy
                                        acc[4][n] += fx * cy * cz;  // xyz
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 5; ++c)
#pragma unroll
                            for (int n = 0; n < NH; ++n)
                                qpart[(qd * 5 + c) * QS + (hh * NH + n) * 32 + lane] = acc[c][n];
                    }
                    epilogue_barrier_or(0);
#pragma unroll
                    for (int xx = 0; xx < XS; ++xx) {
                        const int x = ep * XS + xx;
                        if (x >= G::TX) break;
#pragma unroll
                        for (int c = 0; c < 5; ++c)
                            qall[(5 * r + c) * QS + x * 32 + lane] =
                                ((qpart[(0 * 5 + c) * QS + x * 32 + lane] + qpart[(1 * 5 + c) * QS + x * 32 + lane]) +
                                 qpart[(2 * 5 + c) * QS + x * 32 + lane]) +
                                qpart[(3 * 5 + c) * QS + x * 32 + lane];
                    }
                    epilogue_barrier_or(0);
                }
            } else {
                (void)qall;
            }
            // collision of the quarter's pairs at the lane's TX nodes, pair by pair
            // (FP32: gT_; deviations: dr_ = rho - rho0, gr_ and gb_ the g equilibrium's factor
            // and offset)
            float rho_[G::TX], ux_[G::TX], uy_[G::TX], uz_[G::TX], gT_[G::TX], om_[G::TX], dr_[G::TX], gr_[G::TX],
                gb_[G::TX];
#pragma unroll
            for (int x = 0; x < G::TX; ++x) {
                const float* pn = prm + x * 32 + lane;
                rho_[x] = pn[0 * QS];
                ux_[x] = pn[1 * QS];
                uy_[x] = pn[2 * QS];
                uz_[x] = pn[3 * QS];
                if constexpr (G::kF32) {
                    gT_[x] = pn[4 * QS];
                    om_[x] = pn[5 * QS];
                } else {
                    om_[x] = pn[4 * QS];
                    dr_[x] = pn[5 * QS];
                    gr_[x] = pn[6 * QS];
                    gb_[x] = pn[7 * QS];
                }
            }
            float2* dstp = static_cast<float2*>(a.dst);
            float4* st = stage + ep * 128;
            // Where this lane's store chunks go, as (f, g)-pair offsets inside one velocity's
            // block of the destination (the same for every pair of the tile; -1: a row outside
            // the mesh), and where it reads them in the staging buffer.  (Node offsets stay
            // below 2^31: buffers hold at most 2^31 nodes per velocity.)
            constexpr int RW_ = G::TX * G::PB / 4;
            constexpr bool k16_ = (G::TX * G::PB) % 16 == 0 && (CX * P * G::PB) % 16 == 0;
            constexpr int CW_ = k16_ ? 4 : 2;
            constexpr int NCH_ = RW_ / CW_, NCHP_ = NCH_ | 1;
            constexpr bool kStaged8 = G::kF32 && G::TX == 8;
            constexpr int NI = kStaged8 ? 4 : (G::ROWS * NCH_ + 31) / 32;
            int goff[NI], sidx[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                int r, ch;
                if constexpr (kStaged8) {
                    r = 8 * i + (lane >> 2);
                    ch = lane & 3;
                    sidx[i] = r * 4 + (ch ^ ((r >> 1) & 3));
                } else {
                    const int q = 32 * i + lane;
                    r = q / NCH_;
                    ch = q - r * NCH_;
                    sidx[i] = (r * NCHP_ + ch) * CW_;
                }
                const int oz = r / G::TY, oy = r - (r / G::TY) * G::TY;
                const bool ok = r < G::ROWS && (!kRaggedY || c0[1] * P + oy < a.cells[1] * P);
                goff[i] = ok ? ((c0[2] * P + oz) * a.N[1] + (c0[1] * P + oy)) * a.N[0] + c0[0] * P +
                                   ch * (CW_ * 4 / G::PB)
                             : -1;
            }
            for (int sw = sw0; sw < nsw; ++sw) {
                const int cw = stream_index(qd + 4 * sw), npw = pairs_of(cw);
#pragma unroll 1
                for (int k = 0; k < npw; ++k) {
                    const int j = pair_of(cw, k);
                    float h[2 * G::TX];
                    tmem_load_row<G::TX>(tb + static_cast<uint32_t>(sw * TC::per_warp + k * G::PCS), h);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (sw == nsw - 1 && k == npw - 1) {
                        // the last read of this buffer: hand it back to the stream warps
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tmem_empty0 + 8 * (qd * 2 + bf));
                    }
                    const int sh = shell_of(j);
                    const float xix = t.xi[j][0], xiy = t.xi[j][1], xiz = t.xi[j][2], wj = t.w[j];
                    if constexpr (G::kF32) {
#pragma unroll
                        for (int x = 0; x < G::TX; ++x) {
                            const float* pn = prm + x * 32 + lane;
                            const float sdot = xix * ux_[x] + xiy * uy_[x] + xiz * uz_[x];
                            const float poly =
                                pn[(6 + sh) * QS] +
                                sdot * (pn[(10 + sh) * QS] +
                                        sdot * (pn[(14 + sh) * QS] + sdot * (1.0f / 6.0f + sdot * (1.0f / 24.0f))));
                            const float feq = wj * rho_[x] * poly;
                            const float f = h[2 * x], g = h[2 * x + 1];
                            h[2 * x] = f + om_[x] * (feq - f);
                            h[2 * x + 1] = g + om_[x] * (gT_[x] * feq - g);
                        }
                        if constexpr (PR) {
                            // App. D: f*_i = w_i (Qbar : H3(xi_i)) / 6, g*_i = (2C_v - D) T f*_i,
                            // relaxed at omega - omega_Pr
                            const float* pa = qreg + SM::kQRows * G::TX * 32 + j * 10;
                            float aj[10];
#pragma unroll
                            for (int c = 0; c < 10; ++c) aj[c] = pa[c];
#pragma unroll
                            for (int x = 0; x < G::TX; ++x) {
                                const float* qn = qall + x * 32 + lane;
                                float fw = aj[0] * qn[0];
#pragma unroll
                                for (int c = 1; c < 10; ++c) fw += aj[c] * qn[c * QS];
                                const float fst = wj * fw;
                                const float ompr = prm[18 * QS + x * 32 + lane];
                                h[2 * x] += ompr * fst;
                                h[2 * x + 1] += ompr * gT_[x] * fst;
                            }
                        }
                    } else {
                        // the collision written for the deviations (f^eq / (w rho) - 1 = pm1):
                        //   d'  = d  + omega (rho pm1 + (rho - rho0) - d)
                        //   dg' = dg + omega ((2C_v-D) (T rho pm1 + (T - T0) rho + T0 (rho - rho0)) - dg)
#pragma unroll
                        for (int x = 0; x < G::TX; ++x) {
                            const float* pn = prm + x * 32 + lane;
                            const float sdot = xix * ux_[x] + xiy * uy_[x] + xiz * uz_[x];
                            const float pm1 =
                                pn[(8 + sh) * QS] +
                                sdot * (pn[(12 + sh) * QS] +
                                        sdot * (pn[(16 + sh) * QS] + sdot * (1.0f / 6.0f + sdot * (1.0f / 24.0f))));
                            const float d = h[2 * x], dg = h[2 * x + 1];
                            h[2 * x] = d + om_[x] * (rho_[x] * pm1 + dr_[x] - d);
                            h[2 * x + 1] = dg + om_[x] * (gr_[x] * pm1 + gb_[x] - dg);
                        }
                    }
                    // streaming stores (the new state is not read again in this step, so it
                    // should not push the source boxes' halos out of L2), through the warp's
                    // staging buffer so that each 16-byte store instruction covers 8 whole rows
                    // (64 bytes each) instead of a quarter of 32 rows.  Chunk q of row r sits at
                    // float4 r*4 + (q ^ ((r >> 1) & 3)): both access patterns are free of bank
                    // conflicts.
                    if constexpr (G::kF32 && G::TX == 8) {
                        __syncwarp();
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            st[lane * 4 + (q ^ ((lane >> 1) & 3))] =
                                make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
                        __syncwarp();
                        float2* dj = dstp + static_cast<long long>(j) * a.nn;
#pragma unroll
                        for (int i = 0; i < 4; ++i) __stcs(reinterpret_cast<float4*>(dj + goff[i]), st[sidx[i]]);
                    } else {
                        // the other row widths (FP32 rows of 6 nodes, 16-bit rows of 6 or 8): a
                        // row is NCH chunks of CW 32-bit words (16 bytes where the row's bytes
                        // and its start in the mesh allow it, else 8); lane r puts row r's
                        // chunks into the staging buffer (odd chunk stride per row: no bank
                        // conflicts), then consecutive lanes store consecutive chunks
                        constexpr int RW = G::TX * G::PB / 4;
                        constexpr bool k16 = (G::TX * G::PB) % 16 == 0 && (CX * P * G::PB) % 16 == 0;
                        constexpr int CW = k16 ? 4 : 2;
                        constexpr int NCH = RW / CW, NCHP = NCH | 1;
                        static_assert(RW % CW == 0 && 32 * NCHP * CW * 4 <= 32 * 64, "staging buffer");
                        uint32_t wv[RW];
#pragma unroll
                        for (int x = 0; x < G::TX; ++x) {
                            if constexpr (G::kF32) {
                                wv[2 * x] = __float_as_uint(h[2 * x]);
                                wv[2 * x + 1] = __float_as_uint(h[2 * x + 1]);
                            } else {
                                wv[x] = narrow_pair<S>(h[2 * x], h[2 * x + 1]);
                            }
                        }
                        uint32_t* stw = reinterpret_cast<uint32_t*>(st);
                        __syncwarp();
#pragma unroll
                        for (int q = 0; q < NCH; ++q) {
                            uint32_t* cp = stw + (lane * NCHP + q) * CW;
                            if constexpr (CW == 4)
                                *reinterpret_cast<uint4*>(cp) = make_uint4(wv[4 * q], wv[4 * q + 1], wv[4 * q + 2], wv[4 * q + 3]);
                            else
                                *reinterpret_cast<uint2*>(cp) = make_uint2(wv[2 * q], wv[2 * q + 1]);
                        }
                        __syncwarp();
                        unsigned char* dj = static_cast<unsigned char*>(a.dst) + static_cast<long long>(j) * a.nn * G::PB;
#pragma unroll
                        for (int i = 0; i < NI; ++i) {
                            if (goff[i] < 0) continue;
                            unsigned char* gp = dj + static_cast<long long>(goff[i]) * G::PB;
                            if constexpr (CW == 4)
                                __stcs(reinterpret_cast<uint4*>(gp), *reinterpret_cast<const uint4*>(stw + sidx[i]));
                            else
                                __stcs(reinterpret_cast<uint2*>(gp), *reinterpret_cast<const uint2*>(stw + sidx[i]));
                        }
                    }
                }
            }
        }
    }

    // free the tensor memory once every stream and epilogue warp is done with it
    tc_fence_before();
    consumer_barrier_or(0, (NC + NE) * 32);
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_base_s),
                     "r"(static_cast<uint32_t>(TC::alloc))
                     : "memory");
}

}  // namespace sllbm
