// M2L on the 5th-generation tensor cores: tcgen05.mma kind::tf32 (one TF32 product, or three
// products of hi/lo TF32 parts) or kind::f16 (three products of hi/lo BF16 parts, or FP16 with
// hi/lo parts for the input degrees 0..3 only), FP32 accumulation in TMEM.
//
// The multipole-to-local translation of one level is, for every target box b,
//     L_b = sum_{o in IL(b)} T_o M_{b+o}
// with 189 interaction-list offsets o (well-separated children of the parent's neighbours)
// and level-independent operators T_o in the normalised basis.  Boxes of one octant class c
// (parity of the grid coordinates) share the same 189 offsets, and a source at offset o
// lies in octant class pi = (c + o) mod 2 at sub-grid displacement delta = floor((c+o)/2)
// in {-1,0,1}^3.  Each class is stored as an (n+2)^3 sub-grid with one ghost layer (periodic
// images or zeros) and linearised row-major, so for a fixed (c, pi) every delta is a
// constant row shift  delta_x (n+2)^2 + delta_y (n+2) + delta_z.
//
// A CTA owns 192 consecutive "virtual rows" r0..r0+191 of the target class (interior rows
// are targets, ghost rows are discarded) and accumulates D[coef_out][row] in TMEM:
//   A = T_o chunk      (M = 128 output coefficients x one K chunk of input coefficients), smem
//   B = source slab    (N = 192 rows x the same K chunk) -- one slab per (pi, K chunk) serves
//                      all deltas: the B descriptor just starts delta rows further in.
// Operands are stored in 16-byte core-matrix rows ("cells": 4 TF32 or 8 BF16 coefficients),
// so every mode has the same byte layout; one MMA consumes 32 bytes of K (8 TF32 or 16 BF16).
// Warp 0 streams slabs and operator chunks with cp.async.bulk into a ring of up to 16 stages
// (several lanes issue copies per round); warp 1 issues the MMAs (one elected lane, the loop
// warp-wide); warps 2..9 drain TMEM into the Morton-ordered L.
// Every wait is bounded; on expiry the CTA flags FMM_DEV_TIMEOUT and returns cleanly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <cstring>
#include <vector>

#include "bounds.cuh"
#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmcph {

FMM_BC_TAKE(bc_take_m2l)

namespace {

constexpr int kTcRows = 192;    // default virtual rows (N) per CTA: 280 CTAs = two full waves at depth 5
constexpr int kTcTmemCols = 512; // two accumulators, 256 columns apart
constexpr int kTcAccStride = 256;
constexpr int kTcMaxStages = 16;  // operator-chunk ring depth: as many stages as shared memory holds
constexpr long long kWaitLimit = 4000000000LL;    // clock cycles (about 2 s)
// Operand forms.  K chunk (input coefficients per slab / operator chunk): 16 for TF32, 8 for
// the split 3xTF32 form (hi and lo parts), 16 for the split 3xBF16 form; there a ring stage
// is 8 KB (one operator chunk, all parts) and a slab buffer 64 bytes per row (about 43 KB at
// depth 5), so two slab buffers leave room for a 16-stage ring.
// The FP16 form (kF16mix) works in K steps of 16 coefficients, one product each (11 bits):
// step 0 holds the cross terms of the 8 lowest input coefficients (degrees 0 and 1 and four of
// degree 2) -- A = lo(T) then hi(T), B = hi(M) then lo(M), so that one MMA adds
// lo(T) hi(M) + hi(T) lo(M) -- and steps 1.. the hi parts of all coefficients, 16 per step.
// With the hi hi products of step 1 the lowest coefficients are then carried to about 22 bits.
// The low degrees carry the large monopole and dipole parts of the far field, whose rounding
// the potential and dV/dlambda feel most; a single product for every degree gives TF32-like
// errors (4e-4 in dV/dlambda at 500k atoms), the cross terms of degrees 0 and 1 alone the
// errors of the full three-product split (5e-6).  The steps are grouped three to a chunk (6
// cells, 12 KB stages; the last chunk may hold fewer), so at p = 10 an (operator, shift) is
// 9 MMAs in 3 ring stages: each stage costs the issuer one wait and one commit, and three
// MMAs per stage keep the tensor pipe ahead of that per-stage work.
enum TcMode { kTf32 = 0, kTf32x3 = 1, kBf16x3 = 2, kF16mix = 3 };
template <int MODE>
struct TcCfg {
    static constexpr bool kSplit = MODE == kTf32x3 || MODE == kBf16x3;  // separate lo parts
    static constexpr bool kBf16 = MODE == kBf16x3;
    static constexpr bool kMix = MODE == kF16mix;
    static constexpr bool k16 = kBf16 || kMix;              // 16-bit elements, kind::f16
    static constexpr int kElem = k16 ? 2 : 4;               // bytes per operand element
    static constexpr int kPerCell = 16 / kElem;             // coefficients per 16-byte cell
    static constexpr int kChunk = kMix ? 48 : kBf16 ? 16 : (kSplit ? 8 : 16);
    static constexpr int kKG = kChunk / kPerCell;           // cells per chunk row (4, 2, 2, 6)
    static constexpr int kKSteps = kChunk * kElem / 32;     // MMAs per chunk (32 bytes of K each)
    static constexpr int kParts = kSplit ? 2 : 1;
    static constexpr uint32_t kPartBytes = 128u * kChunk * kElem;  // one operator part (hi or lo)
    static constexpr uint32_t kStageBytes = kParts * kPartBytes;   // 8 KB (12 KB in the FP16 form)
};
// FP16 form: ncp / 16 + 1 K steps (the cross step and the hi steps), three to a chunk.
inline int f16mix_steps(int ncp) { return ncp / 16 + 1; }
inline int f16mix_chunks(int ncp) { return (f16mix_steps(ncp) + 2) / 3; }
inline int f16mix_last_steps(int ncp) { return f16mix_steps(ncp) - 3 * (f16mix_chunks(ncp) - 1); }  // 1, 2 or 3
// First input coefficient of cell j (0..5) of chunk ch: K step s = 3 ch + j / 2, half j % 2;
// at or beyond ncp (steps past the last) the cell holds zeros.
__host__ __device__ inline int f16mix_base(int ch, int j) {
    const int s = 3 * ch + j / 2;
    return s == 0 ? 0 : 16 * (s - 1) + 8 * (j & 1);
}
// which cells hold lo parts (the FP16 rounding of the remainder): in the cross step, the
// first half of the operator (A) and the second half of the multipoles (B)
__host__ __device__ inline bool f16mix_lo_T(int ch, int j) { return ch == 0 && j == 0; }
__host__ __device__ inline bool f16mix_lo_M(int ch, int j) { return ch == 0 && j == 1; }

struct TcLevels {
    int n[kMaxDepth + 1];
    int R[kMaxDepth + 1];
    int S[kMaxDepth + 1];
    long mtc_off[kMaxDepth + 1];  // float offset of the level's packed multipoles
    long l_off[kMaxDepth + 1];    // box offset of the level in L
};

__host__ __device__ inline int dmax_shift(int n) { return (n + 2) * (n + 2) + (n + 2) + 1; }

__device__ __forceinline__ uint32_t spread3_tc(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// The levels packed by one launch: level i covers threads first[i] .. first[i + 1] - 1.
struct PackLevels {
    int nlev;
    int n[kMaxDepth + 1], R[kMaxDepth + 1];
    long first[kMaxDepth + 2];
    long m_off[kMaxDepth + 1];  // float offset of the level in M
    long t_off[kMaxDepth + 1];  // float offset of the level in the packed arrays
};

// Pack every level's multipoles into [class][cell][(n+2)^3 rows][16 bytes] (one launch).  TF32 forms: a cell
// holds 4 coefficients rounded to TF32 (round to nearest: the tensor core itself would
// truncate), and the lo part is the TF32 rounding of the remainder.  BF16 form: a cell holds
// 8 coefficients rounded to BF16 (nearest even), lo = BF16 rounding of the remainder.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {  // a in the low half (first in memory)
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
__device__ __forceinline__ float bf16_lo_of(uint32_t pair) { return __uint_as_float(pair << 16); }
__device__ __forceinline__ float bf16_hi_of(uint32_t pair) { return __uint_as_float(pair & 0xFFFF0000u); }

template <bool BF16>
__global__ void k_m2l_pack(PackLevels pl, int NKG, int ncp, int periodic, const float* __restrict__ M,
                           float* __restrict__ Mtc_all, float* __restrict__ Mtc_lo_all) {
    const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= pl.first[pl.nlev]) return;
    int lv = 0;
    while (lv + 1 < pl.nlev && gt >= pl.first[lv + 1]) ++lv;
    const long tid = gt - pl.first[lv];
    const int n = pl.n[lv], R = pl.R[lv];
    const float* Mlev = M + pl.m_off[lv];
    float* Mtc = Mtc_all + pl.t_off[lv];
    float* Mtc_lo = Mtc_lo_all ? Mtc_lo_all + pl.t_off[lv] : nullptr;
    const int row = (int)(tid % R);
    const int g = (int)((tid / R) % NKG);
    const int cls = (int)(tid / ((long)R * NKG));
    const int m2 = n + 2;
    int i = row / (m2 * m2) - 1, j = (row / m2) % m2 - 1, k = row % m2 - 1;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f), lo = v;
    constexpr int kPerCell = BF16 ? 8 : 4;
    bool ok = kPerCell * g < ncp;
    if (periodic) {
        i = (i + n) % n;
        j = (j + n) % n;
        k = (k + n) % n;
    } else {
        ok = ok && i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n;
    }
    if (ok) {
        const uint32_t box = ((spread3_tc(i) | (spread3_tc(j) << 1) | (spread3_tc(k) << 2)) << 3) | (uint32_t)cls;
        ok = FMM_IN(box, 8L * n * n * n);
    }
    if (ok) {
        const uint32_t box = ((spread3_tc(i) | (spread3_tc(j) << 1) | (spread3_tc(k) << 2)) << 3) | (uint32_t)cls;
        if (BF16) {
            const float4 x0 = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + 8 * g);
            const float4 x1 = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + 8 * g + 4);
            const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            uint32_t hi[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                hi[e] = bf16_pair(xs[2 * e], xs[2 * e + 1]);
                lw[e] = bf16_pair(xs[2 * e] - bf16_lo_of(hi[e]), xs[2 * e + 1] - bf16_hi_of(hi[e]));
            }
            reinterpret_cast<uint4*>(Mtc)[tid] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            reinterpret_cast<uint4*>(Mtc_lo)[tid] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            return;
        }
        const float4 x = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + 4 * g);
        v.x = tc::round_tf32(x.x);
        v.y = tc::round_tf32(x.y);
        v.z = tc::round_tf32(x.z);
        v.w = tc::round_tf32(x.w);
        lo.x = tc::round_tf32(x.x - v.x);
        lo.y = tc::round_tf32(x.y - v.y);
        lo.z = tc::round_tf32(x.z - v.z);
        lo.w = tc::round_tf32(x.w - v.w);
    }
    reinterpret_cast<float4*>(Mtc)[tid] = v;
    if (Mtc_lo) reinterpret_cast<float4*>(Mtc_lo)[tid] = lo;
}

// FP16 form: cells of 8 coefficients rounded to FP16 (nearest even); the lo cells of chunk 0
// hold the FP16 rounding of the remainder.  Coefficients at or beyond ncp are zero.
__device__ __forceinline__ uint32_t f16_pair(float a, float b) {  // a in the low half (first in memory)
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) | ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
}
__global__ void k_m2l_pack_f16mix(PackLevels pl, int NKG, int ncp, int periodic, const float* __restrict__ M,
                                  float* __restrict__ Mtc_all) {
    const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= pl.first[pl.nlev]) return;
    int lv = 0;
    while (lv + 1 < pl.nlev && gt >= pl.first[lv + 1]) ++lv;
    const long tid = gt - pl.first[lv];
    const int n = pl.n[lv], R = pl.R[lv];
    const float* Mlev = M + pl.m_off[lv];
    const int row = (int)(tid % R);
    const int gc = (int)((tid / R) % NKG);
    const int cls = (int)(tid / ((long)R * NKG));
    const int m2 = n + 2;
    int i = row / (m2 * m2) - 1, j = (row / m2) % m2 - 1, k = row % m2 - 1;
    const int ch = gc / 6, cell = gc % 6;
    const int base = f16mix_base(ch, cell);
    bool ok = base < ncp;  // ncp is a multiple of 16: the cell's 8 coefficients all exist
    if (periodic) {
        i = (i + n) % n;
        j = (j + n) % n;
        k = (k + n) % n;
    } else {
        ok = ok && i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n;
    }
    uint4 out = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t box = ((spread3_tc(i) | (spread3_tc(j) << 1) | (spread3_tc(k) << 2)) << 3) | (uint32_t)cls;
    if (ok && FMM_IN(box, 8L * n * n * n)) {
        const float4 x0 = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + base);
        const float4 x1 = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + base + 4);
        float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        if (f16mix_lo_M(ch, cell))
#pragma unroll
            for (int e = 0; e < 8; ++e) xs[e] -= __half2float(__float2half_rn(xs[e]));
        out = make_uint4(f16_pair(xs[0], xs[1]), f16_pair(xs[2], xs[3]), f16_pair(xs[4], xs[5]), f16_pair(xs[6], xs[7]));
    }
    reinterpret_cast<uint4*>(Mtc_all + pl.t_off[lv])[tid] = out;
}

struct TcTile {
    int level, cls, r0, rows;  // rows: the tile's virtual rows (MMA N), a multiple of 16
};

// Warp roles (10 warps): warp 0 = bulk-copy producer, warp 1 = MMA issuer (one elected lane
// issues), warps 2..9 = accumulator drains.  The tensor core aligns addends to the largest and
// truncates, so a long chain of MMAs into one FP32 accumulator drifts; here each source
// class pi and K chunk is accumulated into one of two TMEM accumulators (ping-pong)
// and then added by the drain warps into FP32 registers (round to nearest), which bounds
// every tensor-core chain to one (source class, K chunk) group: at most 27 offsets x 4 K steps
// (x 3 products in the split form).
constexpr int kTcThreads = 320;
constexpr int kTcDrainWarps = 8;

template <int MODE, int ROWS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(const TcTile* __restrict__ tiles, TcLevels lv, const float* __restrict__ Mtc,
             const float* __restrict__ Mtc_lo, const float* __restrict__ Ttc, float* __restrict__ L, int ncp,
             int NKC, int slab_rows, int nstages, int* __restrict__ status, int last_steps, long long wlim) {
    using Cfg = TcCfg<MODE>;
    constexpr bool SPLIT = Cfg::kSplit;
    constexpr int kTcKG = Cfg::kKG;
    constexpr uint32_t kTcTBytes = Cfg::kStageBytes;
    extern __shared__ __align__(1024) uint8_t smem[];
    // two slab buffers, each [part][kgroup][3 ranges][slab_rows][16 B]; range dx+1 holds the source
    // rows r0 + dx (n+2)^2 - (n+3) .. + slab_rows, i.e. every delta_y, delta_z shift of one delta_x
    const uint32_t kg_stride = 3u * (uint32_t)slab_rows * 16u;
    const uint32_t part_bytes = kg_stride * kTcKG;
    const uint32_t slab_bytes = part_bytes * Cfg::kParts;
    uint8_t* slab0 = smem;
    uint8_t* tring = smem + 2 * (size_t)slab_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tring + (size_t)nstages * kTcTBytes);
    uint64_t* slab_full = bars + 0;    // [2]
    // (a slab buffer is free once its group's MMAs have completed, which is the accumulator's
    // acc_full phase of that group, so the producer waits on that; bars + 3 is unused)
    uint64_t* mma_done = bars + 2;     // after an abort: every MMA the issuer issued has completed
    uint64_t* acc_full = bars + 4;     // [2]
    uint64_t* acc_empty = bars + 6;    // [2]
    uint64_t* t_full = bars + 8;                 // [nstages]
    uint64_t* t_empty = bars + 8 + nstages;      // [nstages]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8 + 2 * nstages);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // copies issued (operator chunks, slabs) by the producer and consumed by the MMA issuer,
    // so that after an abort the outstanding copies are waited for before the CTA exits
    volatile int* copy_count = abort_flag + 1;  // [4]: t issued, slabs issued, t taken, slabs taken

    const TcTile tile = tiles[blockIdx.x];
    const int lev = tile.level, c = tile.cls, r0 = tile.r0;
    const int nr = tile.rows;  // this tile's virtual rows (the MMA N): a multiple of 16, at most ROWS
    const int nh = nr >> 1;    // columns per drain half (a multiple of 8)
    const int n = lv.n[lev], R = lv.R[lev];
    const int m2 = n + 2;
    const int NKG = NKC * kTcKG;
    const int ngroups = 8 * NKC;  // (source class, K chunk) groups
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(slab_full + q, 1);
            tc::mbar_init(acc_full + q, 1);
            tc::mbar_init(acc_empty + q, kTcDrainWarps);
        }
        for (int s = 0; s < nstages; ++s) {
            tc::mbar_init(t_full + s, 1);
            tc::mbar_init(t_empty + s, 1);
        }
        tc::mbar_init(mma_done, 1);
        *abort_flag = 0;
        for (int q = 0; q < 4; ++q) copy_count[q] = 0;
        tc::fence_mbar_init();
    }
    if (warp == 2) {
        tc::tmem_alloc(tmem_slot, kTcTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int hal = m2 + 1;  // rows before/after the tile within one delta_x range
    int rs[3], rl[3];
    for (int q = 0; q < 3; ++q) {
        rs[q] = r0 + (q - 1) * m2 * m2 - hal;          // >= 0: r0 >= S = m2^2 + hal
        rl[q] = min(nr + 2 * hal, R - rs[q]);       // > 0:  r0 < R - S
    }
    const float* Mlev = Mtc + lv.mtc_off[lev];
    const float* Mlev_lo = SPLIT ? Mtc_lo + lv.mtc_off[lev] : nullptr;

    if (warp == 0) {
        // ---------------- producer (the whole warp) ----------------
        // One thread issuing one copy at a time cannot keep the MMAs fed: each turn of its loop
        // (waits, barrier arithmetic, copy issue) is a chain of dependent single-thread
        // instructions several hundred cycles long, longer than the MMAs of one operator chunk.
        // So the lanes share the work: in each round, lane r issues the chunk of the r-th next
        // valid offset of the group (up to min(8, ring depth - 1) chunks per round), and a slab load
        // is spread over the lanes as one copy each.  Control flow is warp-uniform; a failed
        // wait in any lane ends the round before anything of it is issued.
        int* sel = const_cast<int*>(copy_count + 4);  // [32]: operator index by rank
        // chunks issued per round: at most half the ring, so that a round is issued while the
        // other half still holds chunks for the MMA issuer (a round waits for the stage of its
        // last chunk, the one nstages back from it)
        const int per_round = max(1, min(8, nstages / 2));
        int t_issued = 0, slabs_issued = 0;
        auto load_slab = [&](int g) {
            const int pi = g / NKC, ch = g % NKC, buf = g & 1;
            uint8_t* dst = slab0 + (size_t)buf * slab_bytes;
            if (lane == 0)
                tc::mbar_arrive_expect_tx(slab_full + buf,
                                          (uint32_t)(rl[0] + rl[1] + rl[2]) * 16u * kTcKG * Cfg::kParts);
            __syncwarp();
            if (lane < 3 * kTcKG) {  // one (cell, delta_x range) per lane
                const int kg = lane / 3, q = lane % 3;
                const int rsq = r0 + (q - 1) * m2 * m2 - hal;
                const int rlq = min(nr + 2 * hal, R - rsq);
                const long e = (((long)pi * NKG + ch * kTcKG + kg) * R + rsq) * 4;
                uint8_t* dq = dst + (size_t)kg * kg_stride + (size_t)q * slab_rows * 16;
                // (a skipped copy ends in the bounded wait of the MMA issuer)
                if (FMM_OK(rsq >= 0 && rlq > 0 && rlq <= slab_rows && rsq + rlq <= R)) {
                    tc::bulk_g2s(dq, Mlev + e, (uint32_t)rlq * 16u, slab_full + buf);
                    if (SPLIT) tc::bulk_g2s(dq + part_bytes, Mlev_lo + e, (uint32_t)rlq * 16u, slab_full + buf);
                }
            }
            ++slabs_issued;
        };
        int base_stage = 0, base_round = 0;  // ring position of chunk t_issued
        bool ok = true;
        load_slab(0);
        for (int g = 0; g < ngroups && ok; ++g) {
            const int pi = g / NKC, ch = g % NKC;
            // the valid shifts of this (target class, source class), in ascending order
            bool valid = false;
            int op_d = 0;
            if (lane < 27) {
                const int ox = 2 * (lane / 9 - 1) + (pi & 1) - cx, oy = 2 * ((lane / 3) % 3 - 1) + ((pi >> 1) & 1) - cy,
                          oz = 2 * (lane % 3 - 1) + ((pi >> 2) & 1) - cz;
                valid = abs(ox) > 1 || abs(oy) > 1 || abs(oz) > 1;
                op_d = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
            }
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            const int cnt = __popc(vmask);
            if (valid) sel[__popc(vmask & ((1u << lane) - 1u))] = op_d;
            __syncwarp();
            // The next group's slab goes into the buffer of group g - 1, free once that group's
            // MMAs have completed: it is issued as soon as the buffer is free, tested (without
            // blocking) between rounds, so that the ring keeps filling meanwhile.
            bool next_issued = g + 1 >= ngroups;
            const int gn = g + 1;
            const uint32_t gn_parity = (uint32_t)(((gn >> 1) - 1) & 1);
            for (int i0 = 0; i0 < cnt; i0 += per_round) {
                if (__shfl_sync(0xffffffffu, *abort_flag, 0)) {  // another role gave up: issue nothing more
                    ok = false;
                    break;
                }
                if (!next_issued) {
                    const bool freed =
                        __shfl_sync(0xffffffffu, gn < 2 || (lane == 0 && tc::mbar_test_wait(acc_full + (gn & 1), gn_parity)), 0);
                    if (freed) {
                        next_issued = true;
                        load_slab(gn);
                    }
                }
                const int nr = min(per_round, cnt - i0);
                const bool mine = lane < nr;
                int stage = base_stage + lane, round = base_round;
                if (stage >= nstages) {
                    stage -= nstages;
                    ++round;
                }
                bool good = true;
                if (mine && t_issued + lane >= nstages)  // the chunk nstages back has been consumed
                    good = tc::mbar_wait_abort(t_empty + stage, (uint32_t)((round - 1) & 1), wlim, abort_flag);
                if (__ballot_sync(0xffffffffu, !good)) {
                    ok = false;
                    break;
                }
                if (mine) {
                    const int op = sel[i0 + lane];
                    tc::mbar_arrive_expect_tx(t_full + stage, kTcTBytes);
                    if (FMM_IN(op, kNumOps))
                        tc::bulk_g2s(tring + (size_t)stage * kTcTBytes, Ttc + ((long)op * NKC + ch) * (kTcTBytes / 4),
                                 kTcTBytes, t_full + stage);  // hi (+ lo) operator chunk
                }
                t_issued += nr;
                base_stage += nr;
                if (base_stage >= nstages) {
                    base_stage -= nstages;
                    ++base_round;
                }
            }
            __syncwarp();  // sel is rewritten by the next group
            if (ok && !next_issued) {
                const bool good = __shfl_sync(
                    0xffffffffu, lane != 0 || tc::mbar_wait_abort(acc_full + (gn & 1), gn_parity, wlim, abort_flag), 0);
                if (!good || __shfl_sync(0xffffffffu, *abort_flag, 0)) {
                    ok = false;
                    break;
                }
                load_slab(gn);
            }
        }
        if (lane == 0) {
            if (!ok) {
                *abort_flag = 1;
                atomicOr(status, FMM_DEV_TIMEOUT);
            }
            copy_count[0] = t_issued;
            copy_count[1] = slabs_issued;
        }
        __syncwarp();
    } else if (warp == 1) {
        {
            // ---------------- MMA issuer (the whole warp; one elected lane issues) ----------------
            // Lean loop: the 27 shifts are unrolled (constant delta), the ring position is a
            // running counter, and the abort flag is only consulted when a wait expires.  Every
            // lane runs the loop so that descriptors and counters stay warp-uniform.
            const uint32_t idesc = Cfg::kMix ? tc::idesc_f16(128, nr)
                                   : Cfg::kBf16 ? tc::idesc_bf16(128, nr) : tc::idesc_tf32(128, nr);
            // descriptors are built once and advanced by adding (byte offset >> 4) to the address field
            const uint64_t a_base = tc::smem_desc_kmajor(tc::smem_u32(tring), 2048u, 128u);
            const uint64_t b_base = tc::smem_desc_kmajor(tc::smem_u32(slab0), kg_stride, 128u);
            int stage = 0;
            uint32_t tphase = 0;
            bool ok = true;
            int t_taken = 0, slabs_taken = 0;
            int* shift_tab = const_cast<int*>(copy_count) + 36;  // [27], after the producer's rank table
            int nshift = 0;
            for (int g = 0; g < ngroups && ok; ++g) {
                const int pi = g / NKC, buf = g & 1;
                // FP16 form: the K steps (one product each) of this group's chunk, 3 but in the last
                const int ch = g % NKC;
                const int mix_kind = !Cfg::kMix ? 0 : ch == NKC - 1 ? last_steps : 3;
                const int qx = (pi & 1) - cx, qy = ((pi >> 1) & 1) - cy, qz = ((pi >> 2) & 1) - cz;
                const int ab = g & 1;
                const uint32_t dacc = tmem + (uint32_t)(ab * kTcAccStride);
                if (g >= 2 && !tc::mbar_wait_all_abort(acc_empty + ab, ((g >> 1) - 1) & 1, wlim, abort_flag)) {
                    ok = false;
                    break;
                }
                if (!tc::mbar_wait_all_abort(slab_full + buf, (g >> 1) & 1, wlim, abort_flag)) {
                    ok = false;
                    break;
                }
                ++slabs_taken;
                tc::fence_after_sync();
                const uint64_t b_buf = b_base + (((uint64_t)buf * slab_bytes) >> 4) + (uint64_t)hal;
                uint32_t acc = 0;
                // the slab row offsets of this (target class, source class)'s valid shifts, in
                // ascending shift order (the order of the producer's copies): built at the first
                // chunk of each source class
                if (ch == 0) {
                    bool valid = false;
                    int off = 0;
                    if (lane < 27) {
                        const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
                        valid = abs(2 * dx + qx) > 1 || abs(2 * dy + qy) > 1 || abs(2 * dz + qz) > 1;
                        off = (dx + 1) * slab_rows + dy * m2 + dz;
                    }
                    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                    nshift = __popc(vmask);
                    __syncwarp();  // the previous group's reads of the table are done
                    if (valid) shift_tab[__popc(vmask & ((1u << lane) - 1u))] = off;
                    __syncwarp();
                }
                // The loop over the valid shifts, kept rolled (a short loop body stays in the
                // instruction cache beside the other roles' code) and specialised per chunk kind
                // so that the issue path of each chunk has no branch on it (the kind is fixed
                // per group).
                auto shifts = [&](auto kind_tag) {
                    constexpr int kKind = decltype(kind_tag)::value;
                    // FP16 form: whether the chunk's stage was seen complete by the probe that
                    // issued with the previous chunk's MMAs (then no wait is needed)
                    bool ready = false;
#pragma unroll 1
                    for (int i = 0; i < nshift; ++i) {
                        const uint64_t bd0 = b_buf + (uint64_t)shift_tab[i];
                        if (!ready && !tc::mbar_wait_all_abort(t_full + stage, tphase, wlim, abort_flag)) return false;
                        ++t_taken;
                        const uint64_t ad0 = a_base + (uint64_t)stage * (kTcTBytes >> 4);
                        int nstage = stage + 1;
                        uint32_t nphase = tphase;
                        if (nstage == nstages) {
                            nstage = 0;
                            nphase ^= 1u;
                        }
                        // the MMAs of this chunk, then the commit that releases its ring stage; one
                        // elected lane issues each K step's products (hi(T) hi(M) + hi(T) lo(M) +
                        // lo(T) hi(M) in the split forms)
                        if (Cfg::kMix) {
                            // A: cells of 2048 bytes (128 rows), a K step = two cells = 4096 bytes;
                            // B: cells kg_stride apart
                            const uint64_t ad1 = ad0 + (4096u >> 4), bd1 = bd0 + ((2u * kg_stride) >> 4);
                            const uint64_t ad2 = ad0 + (8192u >> 4), bd2 = bd0 + ((4u * kg_stride) >> 4);
                            const uint32_t probe = tc::mma_f16_n_probe_w<kKind>(dacc, ad0, bd0, ad1, bd1, ad2, bd2, idesc,
                                                                               acc, t_empty + stage, t_full + nstage, nphase);
                            acc = 1;
                            ready = __all_sync(0xffffffffu, probe != 0u);
                        } else
#pragma unroll
                        for (int ks = 0; ks < Cfg::kKSteps; ++ks) {  // 32 bytes of K = two cells per MMA
                            const uint64_t ad = ad0 + (uint64_t)ks * (4096u >> 4);
                            const uint64_t bd = bd0 + (uint64_t)ks * ((2u * kg_stride) >> 4);
                            const bool last_ks = ks == Cfg::kKSteps - 1;
                            if (SPLIT) {
                                if (last_ks)
                                    tc::mma3_w<Cfg::kBf16, true>(dacc, ad, bd, ad + (Cfg::kPartBytes >> 4),
                                                                 bd + (part_bytes >> 4), idesc, acc, t_empty + stage);
                                else
                                    tc::mma3_w<Cfg::kBf16, false>(dacc, ad, bd, ad + (Cfg::kPartBytes >> 4),
                                                                  bd + (part_bytes >> 4), idesc, acc, nullptr);
                            } else {
                                if (last_ks)
                                    tc::mma1_tf32_w<true>(dacc, ad, bd, idesc, acc, t_empty + stage);
                                else
                                    tc::mma1_tf32_w<false>(dacc, ad, bd, idesc, acc, nullptr);
                            }
                            acc = 1;
                        }
                        stage = nstage;
                        tphase = nphase;
                    }
                    return true;
                };
                if (!Cfg::kMix || mix_kind == 3) ok = shifts(std::integral_constant<int, 3>{});
                else if (mix_kind == 2) ok = shifts(std::integral_constant<int, 2>{});
                else ok = shifts(std::integral_constant<int, 1>{});
                if (!ok) break;
                tc::mma_commit_w(acc_full + ab);  // this group's partial sum is complete, its slab free
            }
            if (!ok && lane == 0) {
                // Give up: no more MMAs.  The other roles see the flag in their waits (nothing
                // completes a barrier phase without the work behind it, so the producer never
                // reuses a buffer whose copy has not been consumed).
                *abort_flag = 1;
                atomicOr(status, FMM_DEV_TIMEOUT);
            }
            // Every path: wait (with the full bound) until every MMA issued has completed, so
            // that none is still reading shared memory or writing TMEM when the CTA frees them --
            // also when a drain warp gave up after the last group was issued.  Normally this
            // completes with the last group's accumulator, which the drains wait for anyway.
            tc::mma_commit_w(mma_done);
            tc::mbar_wait_all(mma_done, 0, kWaitLimit);
            if (lane == 0) {
                copy_count[2] = t_taken;
                copy_count[3] = slabs_taken;
            }
        }
        __syncwarp();
    } else {
        // ---------------- accumulator drains (warps 2..9) ----------------
        const int q = warp & 3;                    // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;          // column half of the tile
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        float sum[ROWS / 2];
#pragma unroll
        for (int i = 0; i < ROWS / 2; ++i) sum[i] = 0.f;
        bool ok = true;
        for (int grp = 0; grp < ngroups; ++grp) {
            const int ab = grp & 1;
            if (!tc::mbar_wait_backoff_abort(acc_full + ab, (grp >> 1) & 1, wlim, abort_flag) || *abort_flag) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t base = tmem + lane_base + (uint32_t)(ab * kTcAccStride + half * nh);
#pragma unroll
            for (int cb = 0; cb < ROWS / 2; cb += 16) {  // nh is warp-uniform: the loads stay aligned
                if (cb + 16 <= nh) {
                    float v[16];
                    tc::tmem_ld16(base + cb, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) sum[cb + e] += v[e];
                } else if (cb + 8 <= nh) {
                    float v[8];
                    tc::tmem_ld8(base + cb, v);
#pragma unroll
                    for (int e = 0; e < 8; ++e) sum[cb + e] += v[e];
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acc_empty + ab);
        }
        if (ok && !*abort_flag) {
            // The nh rows of this half go to their Morton boxes: first a table of the rows' box
            // offsets in shared memory (the operator ring is idle: every MMA has completed), three
            // rows per lane, then one store per row.  A fully unrolled loop doing the index
            // arithmetic per row is long straight-line code that runs once per tile, mostly
            // waiting for instruction fetch.
            int* tab = reinterpret_cast<int*>(tring) + (warp - 2) * (ROWS / 2);
            const int rfirst = r0 + half * nh;
            for (int e = lane; e < nh; e += 32) {
                const int r = rfirst + e;
                const int ip = r / (m2 * m2), jp = (r / m2) % m2, kp = r % m2;
                int off = -1;
                if (r < R && ip >= 1 && ip <= n && jp >= 1 && jp <= n && kp >= 1 && kp <= n)
                    off = (int)(((spread3_tc(ip - 1) | (spread3_tc(jp - 1) << 1) | (spread3_tc(kp - 1) << 2)) << 3) |
                                (uint32_t)c) * ncp;
                if (off >= 0 && !FMM_IN(off / ncp, 8L * n * n * n)) off = -1;
                tab[e] = off;
            }
            __syncwarp();
            const int j = q * 32 + lane;  // output coefficient = TMEM lane
            float* Ll = L + lv.l_off[lev] * (long)ncp + j;
            if (j < ncp) {
#pragma unroll
                for (int e = 0; e < ROWS / 2; ++e) {
                    const int off = e < nh ? tab[e] : -1;
                    if (off >= 0) Ll[off] = sum[e];
                }
            }
        } else if (lane == 0) {
            *abort_flag = 1;
            atomicOr(status, FMM_DEV_TIMEOUT);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0 && lane == 0 && *abort_flag) {
        // copies issued but never consumed may still be landing in shared memory: wait for them
        // (bounded) before the CTA exits; ring use j is stage j % nstages with phase parity
        // (j / nstages) & 1
        for (int j = copy_count[2]; j < copy_count[0]; ++j)
            tc::mbar_wait(t_full + j % nstages, (uint32_t)((j / nstages) & 1), kWaitLimit);
        for (int g = copy_count[3]; g < copy_count[1]; ++g)
            tc::mbar_wait(slab_full + (g & 1), (uint32_t)((g >> 1) & 1), kWaitLimit);
    }
    __syncthreads();
    if (warp == 2) tc::tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace

// The tile widths (virtual rows per CTA, the MMA N) the kernel is instantiated for.
template <class F>
void for_tile_rows(F&& f) {
    f(std::integral_constant<int, 128>{});
    f(std::integral_constant<int, 160>{});
    f(std::integral_constant<int, 176>{});
    f(std::integral_constant<int, 192>{});
    f(std::integral_constant<int, 224>{});
    f(std::integral_constant<int, 256>{});
}
bool m2l_tile_rows_ok(int rows) {
    return rows == 0 || rows == 128 || rows == 160 || rows == 176 || rows == 192 || rows == 224 || rows == 256;
}

// ------------------------------------------------------------------------------------------
struct TcState {
    int mode = kTf32;
    float* Mtc_lo = nullptr;
    float* Mtc = nullptr;
    float* Ttc = nullptr;
    TcTile* tiles = nullptr;
    int ntiles = 0;
    int tile_first[kMaxDepth + 2] = {};  // the tiles of level l are [tile_first[l], tile_first[l + 1])
    int NKC = 0;
    int last_steps = 3;  // FP16 form: K steps in the last chunk (1..3)
    int KG = 0;  // 16-byte cells per K chunk
    int slab_rows = 0;
    int rows = kTcRows;  // widest tile (MMA N) per CTA: 128, 160, 176, 192, 224 or 256
    int nstages = 0;  // operator ring depth
    size_t smem = 0;
    TcLevels lv{};
};

bool m2l_tc_supported(const Handle* h) {
    // M = 128 output coefficients per MMA; the slab of the deepest level fits in shared memory
    const bool mixed = h->precision == FMM_MIXED_TF32 || h->precision == FMM_MIXED_3XTF32 ||
                       h->precision == FMM_MIXED_3XBF16 || h->precision == FMM_MIXED_FP16;
    return mixed && h->ncp <= 128 && h->depth <= 5;
}

static TcState* tc_state(Handle* h) { return reinterpret_cast<TcState*>(h->tc); }

namespace {
// Host roundings of the operator parts, matching the device packing of the multipoles.
float host_tf32(float x) {  // nearest, ties away from zero (cvt.rna.tf32.f32)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}
uint16_t host_bf16_bits(float x) {  // nearest, ties to even (cvt.rn.bf16.f32); finite inputs
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float host_bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

template <int MODE>
void pack_operators(const std::vector<float>& Trm, int nc, int NKC, std::vector<uint8_t>& out) {
    using Cfg = TcCfg<MODE>;
    // [op][chunk][part][cell][j (128)][16 bytes]; part 0 = hi rounding, part 1 = rounding of the remainder
    out.assign((size_t)kNumOps * NKC * Cfg::kStageBytes, 0);
    for (int op = 0; op < kNumOps; ++op)
        for (int jj = 0; jj < nc; ++jj)
            for (int k = 0; k < nc; ++k) {
                const float v = Trm[((size_t)op * nc + jj) * nc + k];
                const int ch = k / Cfg::kChunk, g = (k % Cfg::kChunk) / Cfg::kPerCell, e = k % Cfg::kPerCell;
                for (int part = 0; part < Cfg::kParts; ++part) {
                    const size_t cell = ((((size_t)op * NKC + ch) * Cfg::kParts + part) * Cfg::kKG + g) * 128 + jj;
                    uint8_t* dst = out.data() + cell * 16 + (size_t)e * Cfg::kElem;
                    if (Cfg::kBf16) {
                        const uint16_t hi = host_bf16_bits(v);
                        const uint16_t w = part == 0 ? hi : host_bf16_bits(v - host_bf16_value(hi));
                        std::memcpy(dst, &w, 2);
                    } else {
                        const float hi = host_tf32(v);
                        const float w = part == 0 ? hi : host_tf32(v - hi);
                        std::memcpy(dst, &w, 4);
                    }
                }
            }
}
// FP16 form: [op][chunk][cell j (6)][128 rows][16 bytes], cell j of chunk ch holding the
// coefficients f16mix_base(ch, j) .. + 7 (hi part, or for the lo cell of the cross step the
// FP16 rounding of the remainder), zero at or beyond nc.
void pack_operators_f16mix(const std::vector<float>& Trm, int nc, int NKC, std::vector<uint8_t>& out) {
    out.assign((size_t)kNumOps * NKC * TcCfg<kF16mix>::kStageBytes, 0);
    for (int op = 0; op < kNumOps; ++op)
        for (int ch = 0; ch < NKC; ++ch)
            for (int j = 0; j < 6; ++j) {
                const int base = f16mix_base(ch, j);
                for (int jj = 0; jj < nc; ++jj)
                    for (int e = 0; e < 8 && base + e < nc; ++e) {
                        const float v = Trm[((size_t)op * nc + jj) * nc + base + e];
                        const __half hi = __float2half_rn(v);
                        const __half w = f16mix_lo_T(ch, j) ? __float2half_rn(v - __half2float(hi)) : hi;
                        const size_t cell = (((size_t)op * NKC + ch) * 6 + j) * 128 + jj;
                        std::memcpy(out.data() + cell * 16 + (size_t)e * 2, &w, 2);
                    }
            }
}
}  // namespace

int m2l_tc_setup(Handle* h, const std::vector<float>& T_rowmajor /*[343][nc][nc] j-major*/) {
    TcState* st = new TcState();
    h->tc = st;
    const int nc = h->nc, ncp = h->ncp, d = h->depth;
    st->rows = h->m2l_rows > 0 ? h->m2l_rows : kTcRows;
    st->mode = h->precision == FMM_MIXED_3XTF32 ? kTf32x3
               : h->precision == FMM_MIXED_3XBF16 ? kBf16x3
               : h->precision == FMM_MIXED_FP16   ? kF16mix
                                                  : kTf32;
    int chunk = 0, nparts = 1;
    uint32_t stage_bytes = 0;
    std::vector<uint8_t> T;
    switch (st->mode) {
        case kTf32x3:
            chunk = TcCfg<kTf32x3>::kChunk, st->KG = TcCfg<kTf32x3>::kKG, nparts = 2;
            stage_bytes = TcCfg<kTf32x3>::kStageBytes;
            st->NKC = (ncp + chunk - 1) / chunk;
            pack_operators<kTf32x3>(T_rowmajor, nc, st->NKC, T);
            break;
        case kBf16x3:
            chunk = TcCfg<kBf16x3>::kChunk, st->KG = TcCfg<kBf16x3>::kKG, nparts = 2;
            stage_bytes = TcCfg<kBf16x3>::kStageBytes;
            st->NKC = (ncp + chunk - 1) / chunk;
            pack_operators<kBf16x3>(T_rowmajor, nc, st->NKC, T);
            break;
        case kF16mix:
            st->KG = TcCfg<kF16mix>::kKG, nparts = 1;
            stage_bytes = TcCfg<kF16mix>::kStageBytes;
            st->NKC = f16mix_chunks(ncp);
            st->last_steps = f16mix_last_steps(ncp);
            pack_operators_f16mix(T_rowmajor, nc, st->NKC, T);
            break;
        default:
            chunk = TcCfg<kTf32>::kChunk, st->KG = TcCfg<kTf32>::kKG, nparts = 1;
            stage_bytes = TcCfg<kTf32>::kStageBytes;
            st->NKC = (ncp + chunk - 1) / chunk;
            pack_operators<kTf32>(T_rowmajor, nc, st->NKC, T);
    }
    const int NKG = st->NKC * st->KG;
    // packed multipole levels
    long off = 0;
    for (int l = 0; l <= kMaxDepth; ++l) {
        st->lv.n[l] = st->lv.R[l] = st->lv.S[l] = 0;
        st->lv.mtc_off[l] = 0;
        st->lv.l_off[l] = 0;
    }
    std::vector<TcTile> tiles;
    for (int l = 0; l <= kMaxDepth + 1; ++l) st->tile_first[l] = 0;
    for (int l = h->lmin; l <= d; ++l) {
        st->tile_first[l] = (int)tiles.size();
        const int n = 1 << (l - 1);
        const int R = (n + 2) * (n + 2) * (n + 2);
        const int S = dmax_shift(n);
        st->lv.n[l] = n;
        st->lv.R[l] = R;
        st->lv.S[l] = S;
        st->lv.mtc_off[l] = off;
        st->lv.l_off[l] = h->lvl_off[l];
        off += 8L * NKG * R * 4;  // 16-byte cells, counted in floats
        // target rows S .. R - S - 1 in k tiles of equal width (a multiple of 16, at most the
        // launch's width): at the coarse levels a tile is only as wide as its level needs
        const int range = R - 2 * S;
        const int k = (range + st->rows - 1) / st->rows;
        const int w = std::min(st->rows, 16 * (((range + k - 1) / k + 15) / 16));
        for (int c = 0; c < 8; ++c)
            for (int r0 = S; r0 < R - S; r0 += w) tiles.push_back({l, c, r0, w});
    }
    for (int l = d + 1; l <= kMaxDepth + 1; ++l) st->tile_first[l] = (int)tiles.size();
    st->slab_rows = st->rows + 2 * ((1 << (d - 1)) + 3);  // one delta_x range at the deepest level
    // two slab buffers, then as many ring stages as fit (at least 3), then barriers and flags
    constexpr size_t kBarBytes = 1024;  // barriers, TMEM slot, flags, copy counts, rank and shift tables
    const size_t slabs = 2 * (size_t)3 * st->slab_rows * st->KG * 16 * nparts;
    const size_t room = 227 * 1024 > slabs + kBarBytes ? 227 * 1024 - slabs - kBarBytes : 0;
    st->nstages = std::max(3, std::min(kTcMaxStages, (int)(room / stage_bytes)));
    st->smem = slabs + (size_t)st->nstages * stage_bytes + kBarBytes;
    st->ntiles = (int)tiles.size();
    if (device_alloc((void**)&st->Ttc, T.size()) != cudaSuccess ||
        device_alloc((void**)&st->Mtc, sizeof(float) * (off > 0 ? off : 4)) != cudaSuccess ||
        (nparts == 2 && device_alloc((void**)&st->Mtc_lo, sizeof(float) * (off > 0 ? off : 4)) != cudaSuccess) ||
        device_alloc((void**)&st->tiles, sizeof(TcTile) * (tiles.empty() ? 1 : tiles.size())) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ERR_OOM;
    }
    cudaMemcpy(st->Ttc, T.data(), T.size(), cudaMemcpyHostToDevice);
    if (!tiles.empty()) cudaMemcpy(st->tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice);
    if (st->smem > 227 * 1024) return FMM_ERR_ARG;
    // The attribute is process wide per kernel: set it to the per-block maximum once, so that
    // handles of different depths (different slab sizes) never lower each other's limit.
    constexpr int kMaxDynSmem = 227 * 1024;
    for_tile_rows([&](auto rows_tag) {
        constexpr int R = decltype(rows_tag)::value;
        cudaFuncSetAttribute(k_m2l_tc<kTf32, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        cudaFuncSetAttribute(k_m2l_tc<kTf32x3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        cudaFuncSetAttribute(k_m2l_tc<kBf16x3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        cudaFuncSetAttribute(k_m2l_tc<kF16mix, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    });
    return FMM_OK;
}

void m2l_tc_free(Handle* h) {
    TcState* st = tc_state(h);
    if (!st) return;
    if (st->Mtc) cudaFree(st->Mtc);
    if (st->Mtc_lo) cudaFree(st->Mtc_lo);
    if (st->Ttc) cudaFree(st->Ttc);
    if (st->tiles) cudaFree(st->tiles);
    delete st;
    h->tc = nullptr;
}

int m2l_tc_launches(const Handle* h) {
    return 2;  // per call of launch_m2l_tc: the pack of its levels + the MMA kernel
}

void launch_m2l_tc(Handle* h, cudaStream_t stream, int lo, int hi, int parts) {
    TcState* st = tc_state(h);
    const int NKG = st->NKC * st->KG;
    const bool bf16 = st->mode == kBf16x3;
    lo = std::max(lo, h->lmin);
    hi = std::min(hi, h->depth);
    if (lo > hi) return;
    PackLevels pl{};
    long tot = 0;
    for (int l = lo; l <= hi; ++l) {
        const int i = pl.nlev++;
        pl.n[i] = st->lv.n[l];
        pl.R[i] = st->lv.R[l];
        pl.first[i] = tot;
        pl.m_off[i] = h->lvl_off[l] * h->ncp;
        pl.t_off[i] = st->lv.mtc_off[l];
        tot += 8L * NKG * st->lv.R[l];
    }
    pl.first[pl.nlev] = tot;
    if (tot > 0 && (parts & kM2lPack)) {
        const unsigned grid = (unsigned)((tot + 255) / 256);
        if (st->mode == kF16mix)
            k_m2l_pack_f16mix<<<grid, 256, 0, stream>>>(pl, NKG, h->ncp, h->periodic, h->M, st->Mtc);
        else if (bf16)
            k_m2l_pack<true><<<grid, 256, 0, stream>>>(pl, NKG, h->ncp, h->periodic, h->M, st->Mtc, st->Mtc_lo);
        else
            k_m2l_pack<false><<<grid, 256, 0, stream>>>(pl, NKG, h->ncp, h->periodic, h->M, st->Mtc, st->Mtc_lo);
    }
    const int t0 = st->tile_first[lo], nt = st->tile_first[hi + 1] - t0;
    if (nt <= 0 || !(parts & kM2lMma)) return;
    const long long wlim = h->wait_limit > 0 ? h->wait_limit : kWaitLimit;
    const TcTile* tiles = st->tiles + t0;
    auto launch = [&](auto rows_tag) {
        constexpr int R = decltype(rows_tag)::value;
        if (R != st->rows) return;
        switch (st->mode) {
            case kTf32x3:
                k_m2l_tc<kTf32x3, R><<<nt, kTcThreads, st->smem, stream>>>(
                    tiles, st->lv, st->Mtc, st->Mtc_lo, st->Ttc, h->L, h->ncp, st->NKC, st->slab_rows, st->nstages,
                    h->status, 0, wlim);
                break;
            case kBf16x3:
                k_m2l_tc<kBf16x3, R><<<nt, kTcThreads, st->smem, stream>>>(
                    tiles, st->lv, st->Mtc, st->Mtc_lo, st->Ttc, h->L, h->ncp, st->NKC, st->slab_rows, st->nstages,
                    h->status, 0, wlim);
                break;
            case kF16mix:
                k_m2l_tc<kF16mix, R><<<nt, kTcThreads, st->smem, stream>>>(
                    tiles, st->lv, st->Mtc, nullptr, st->Ttc, h->L, h->ncp, st->NKC, st->slab_rows, st->nstages,
                    h->status, st->last_steps, wlim);
                break;
            default:
                k_m2l_tc<kTf32, R><<<nt, kTcThreads, st->smem, stream>>>(
                    tiles, st->lv, st->Mtc, nullptr, st->Ttc, h->L, h->ncp, st->NKC, st->slab_rows, st->nstages,
                    h->status, 0, wlim);
        }
    };
    for_tile_rows(launch);
}

}  // namespace fmmcph
