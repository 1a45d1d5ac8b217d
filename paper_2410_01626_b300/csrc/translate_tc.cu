// M2M and L2L on the 5th-generation tensor cores, split TF32 (hi*hi + hi*lo + lo*hi, about 22
// significant bits per operand), FP32 accumulation in TMEM.  The split is TF32 rather than
// BF16 here: these products run at every level on the same coarse expansions, so their
// operand rounding is coherent across large regions instead of averaging out as in M2L, and
// the products are small enough that the tensor rate does not matter.
//
// Both translations of one level are one product with a fixed, level-independent operator W
// (the normalised basis makes it so) and the expansions X of one level:
//   M2M: M_parent[p][j]        = sum_{c,k} W[j][(c,k)] M_child[8p + c][k]   (K = 8 ncp)
//   L2L: L_child[8p + c][j]   += sum_k W[(c,j)][k] L_parent[p][k]          (K = ncp)
// i.e. D[m][p] = sum_k W[m][k] X[p][k] with X rows p of K contiguous floats (the 8 children of
// a parent are contiguous in Morton order) and the result written to C[p * ldc + m].
// A CTA owns 128 rows m (one MMA M) x 128 boxes p (N) and a slice of K: W arrives by bulk copy
// (pre-packed on the host as hi/lo TF32 in core-matrix cells), X is loaded by the 128 threads
// (one box row each), split into hi/lo TF32 and stored in the same cell layout.  Two stages
// alternate so that the loads of one K chunk overlap the MMAs of the previous one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "bounds.cuh"
#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmcph {

FMM_BC_TAKE(bc_take_translate)

namespace {

constexpr int kGThreads = 256;  // two threads per box row: latency-bound code gets more issue slots
constexpr int kGRows = 128;               // M per CTA (one MMA)
constexpr int kGBoxes = 128;              // N per CTA
constexpr int kGChunk = 16;               // K coefficients per stage
constexpr int kGCells = kGChunk / 4;      // 16-byte cells (4 TF32) per row and stage
constexpr uint32_t kGPart = kGRows * kGChunk * 4;  // one hi or lo part of a stage operand: 8 KB
constexpr uint32_t kGStage = 2 * kGPart;           // hi + lo: 16 KB
constexpr long long kGWaitLimit = 4000000000LL;    // clock cycles (about 2 s): the default
                                                   // pipeline limit, and always that of the
                                                   // drains after an abort
constexpr size_t kGSmem = 2 * (size_t)kGStage * 2 + 1024;  // two stages of W and X, barriers


// grid: (N tiles, M tiles, K slices).  Slice z covers chunks [z kps, (z + 1) kps) and writes
// C + z cstride; accumulate adds to C instead of overwriting it.  wlim bounds the pipeline's
// waits (clock cycles); when one expires the CTA stops issuing, waits for what it issued, sets
// FMM_DEV_TIMEOUT and writes nothing.  lose_copies (a test hook, fmm_inject_copy_loss): the W
// copies are announced on their barrier but not issued.
__global__ void __launch_bounds__(kGThreads, 1)
    k_translate_tc(const uint8_t* __restrict__ Wp, int Mtot, int nkc, int K, const float* __restrict__ X, int ldx,
                   int N, float* __restrict__ C, int ldc, int accumulate, int kps, long cstride,
                   int* __restrict__ status, long long wlim, int lose_copies) {
    extern __shared__ __align__(1024) uint8_t gsm[];
    uint8_t* wst = gsm;                       // [2 stages][hi, lo][cell][128 rows][16 B]
    uint8_t* xst = gsm + 2 * (size_t)kGStage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + 4 * (size_t)kGStage);
    uint64_t* w_full = bars;        // [2]
    uint64_t* mma_done = bars + 2;  // [2]
    uint64_t* acc_done = bars + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int n0 = blockIdx.x * kGBoxes, mt = blockIdx.y, z = blockIdx.z;
    const int kc0 = z * kps, kc1 = min(nkc, kc0 + kps);
    C += (long)z * cstride;
    if (t == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(w_full + s, 1);
            tc::mbar_init(mma_done + s, 1);
        }
        tc::mbar_init(acc_done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, kGBoxes);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::idesc_tf32(kGRows, kGBoxes);
    const uint64_t wdesc0 = tc::smem_desc_kmajor(tc::smem_u32(wst), 2048u, 128u);
    const uint64_t xdesc0 = tc::smem_desc_kmajor(tc::smem_u32(xst), 2048u, 128u);
    const int row = t & (kGBoxes - 1), half = t / kGBoxes;  // this thread's box row of X, half of its cells
    constexpr int kHalfCells = kGCells / 2;
    const int p = n0 + row;
    const int nch = kc1 - kc0;
    auto load_x = [&](int kc, float4* xv) {
#pragma unroll
        for (int gg = 0; gg < kHalfCells; ++gg) {
            const int g = half * kHalfCells + gg;
            const int k = kc * kGChunk + g * 4;
            xv[gg] = (p < N && k < K) ? *reinterpret_cast<const float4*>(X + (long)p * ldx + k)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    int w_issued = 0, w_taken = 0;  // W chunks copied / consumed (thread 0)
    auto issue_w = [&](int i) {  // W chunk kc0 + i into stage i & 1 (thread 0)
        const int s = i & 1;
        tc::mbar_arrive_expect_tx(w_full + s, kGStage);
        if (lose_copies) return;  // test hook: announced, never issued, so the wait runs out
        ++w_issued;
        if (FMM_IN((long)mt * nkc + kc0 + i, (long)((Mtot + kGRows - 1) / kGRows) * nkc))  // (else the bounded wait)
            tc::bulk_g2s(wst + (size_t)s * kGStage, Wp + ((size_t)mt * nkc + kc0 + i) * kGStage, kGStage, w_full + s);
    };
    float4 xv[kHalfCells], xn[kHalfCells];
    if (nch > 0) {
        load_x(kc0, xv);
        if (t == 0) issue_w(0);
    }
    for (int i = 0; i < nch; ++i) {
        const int s = i & 1;
        // stage s is free once the MMAs of chunk i - 2 have completed; every thread waits, and
        // the abort decision is taken by all threads together after the barrier
        if (i >= 2 && !tc::mbar_wait(mma_done + s, ((i >> 1) - 1) & 1, wlim)) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) break;
        if (i + 1 < nch) load_x(kc0 + i + 1, xn);  // next chunk's rows, in flight during this one
        // X chunk i: split into hi / lo TF32 cells (round to nearest: the tensor core itself
        // would truncate)
        uint8_t* xs = xst + (size_t)s * kGStage;
#pragma unroll
        for (int gg = 0; gg < kHalfCells; ++gg) {
            const int g = half * kHalfCells + gg;
            const float4 v = xv[gg];
            const float4 hi = make_float4(tc::round_tf32(v.x), tc::round_tf32(v.y), tc::round_tf32(v.z),
                                          tc::round_tf32(v.w));
            const float4 lo = make_float4(tc::round_tf32(v.x - hi.x), tc::round_tf32(v.y - hi.y),
                                          tc::round_tf32(v.z - hi.z), tc::round_tf32(v.w - hi.w));
            *reinterpret_cast<float4*>(xs + (size_t)g * 2048 + (size_t)row * 16) = hi;
            *reinterpret_cast<float4*>(xs + kGPart + (size_t)g * 2048 + (size_t)row * 16) = lo;
        }
        tc::fence_proxy_async();  // the generic-proxy stores above, for the tensor core
        __syncthreads();
        if (t == 0) {
            if (!tc::mbar_wait(w_full + s, (i >> 1) & 1, wlim)) {
                *abort_flag = 1;
            } else {
                ++w_taken;
                tc::fence_after_sync();
                const uint64_t wd = wdesc0 + (((uint64_t)s * kGStage) >> 4);
                const uint64_t xd = xdesc0 + (((uint64_t)s * kGStage) >> 4);
#pragma unroll
                for (int ks = 0; ks < kGChunk / 8; ++ks) {  // 8 TF32 = two cells per MMA
                    const uint64_t a = wd + (uint64_t)ks * (4096u >> 4), b = xd + (uint64_t)ks * (4096u >> 4);
                    tc::mma_tf32(tmem, a, b, idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, a, b + (kGPart >> 4), idesc, 1u);
                    tc::mma_tf32(tmem, a + (kGPart >> 4), b, idesc, 1u);
                }
                tc::mma_commit(mma_done + s);
                // the next W chunk goes to the other stage once the MMAs of chunk i - 1 are done
                if (i + 1 < nch) {
                    if (i >= 1 && !tc::mbar_wait(mma_done + (s ^ 1), ((i - 1) >> 1) & 1, wlim))
                        *abort_flag = 1;
                    else
                        issue_w(i + 1);
                }
            }
        }
#pragma unroll
        for (int gg = 0; gg < kHalfCells; ++gg) xv[gg] = xn[gg];
    }
    __syncthreads();
    const bool ok = *abort_flag == 0;
    if (t == 0) {
        // after an abort, no bulk copy may still be writing this CTA's shared memory
        for (int i = w_taken; i < w_issued; ++i) tc::mbar_wait(w_full + (i & 1), (i >> 1) & 1, kGWaitLimit);
        tc::mma_commit(acc_done);  // completes once every MMA issued above has
    }
    const bool done = tc::mbar_wait(acc_done, 0, kGWaitLimit);
    if (ok && done && kc1 > kc0) {
        tc::fence_after_sync();
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (the rows), warps 0-3 the first half of the
        // columns (boxes) and warps 4-7 the second
        const int q = warp & 3;
        const int m = mt * kGRows + q * 32 + lane;
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16);
        // a rolled loop: this epilogue runs once per CTA, and unrolled it is long straight-line
        // code that mostly waits for instruction fetch
#pragma unroll 1
        for (int cb = half * (kGBoxes / 2); cb < (half + 1) * (kGBoxes / 2); cb += 16) {
            float v[16];
            tc::tmem_ld16(base + cb, v);
            if (m < Mtot) {
                float old[16];
                if (accumulate) {  // all 16 loads in flight before any store
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int pp = n0 + cb + e;
                        old[e] = pp < N ? C[(long)pp * ldc + m] : 0.f;
                    }
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int pp = n0 + cb + e;
                    if (pp < N) C[(long)pp * ldc + m] = accumulate ? old[e] + v[e] : v[e];
                }
            }
        }
    } else if (!(ok && done) && t == 0) {
        atomicOr(status, FMM_DEV_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kGBoxes);
}

// C (=|+=) sum_z P_z over the split-K partial products, in slice order
__global__ void k_translate_sum(int N, int ldc, int nz, const float* __restrict__ P, long pstride,
                                float* __restrict__ C, int accumulate) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)N * ldc) return;
    const float c0 = accumulate ? C[e] : 0.f;
    float s = 0.f;
    int z = 0;
    for (; z + 8 <= nz; z += 8) {  // eight loads in flight, then the adds in slice order
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = P[(z + k) * pstride + e];
#pragma unroll
        for (int k = 0; k < 8; ++k) s += v[k];
    }
    for (; z < nz; ++z) s += P[z * pstride + e];
    C[e] = accumulate ? c0 + s : s;
}

float tf32_rna(float x) {  // nearest, ties away from zero (cvt.rna.tf32.f32); finite inputs
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

}  // namespace

// W row-major [Mtot][K] -> [m tile][k chunk][hi, lo][cell][128 rows][4 TF32], zero padded.
TranslateOp translate_pack(const std::vector<float>& W, int Mtot, int K) {
    TranslateOp op;
    op.Mtot = Mtot;
    op.K = K;
    op.nmt = (Mtot + kGRows - 1) / kGRows;
    op.nkc = (K + kGChunk - 1) / kGChunk;
    std::vector<float> P((size_t)op.nmt * op.nkc * kGStage / 4, 0.f);
    for (int m = 0; m < Mtot; ++m)
        for (int k = 0; k < K; ++k) {
            const float v = W[(size_t)m * K + k];
            const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
            const int mt = m / kGRows, r = m % kGRows, kc = k / kGChunk, g = (k % kGChunk) / 4, e = k % 4;
            const size_t cell = (((size_t)mt * op.nkc + kc) * 2 * kGCells + g) * kGRows + r;  // part 0
            P[cell * 4 + e] = hi;
            P[(cell + (size_t)kGCells * kGRows) * 4 + e] = lo;  // part 1: kGCells cells further
        }
    op.bytes = P.size() * 4;
    if (device_alloc((void**)&op.dev, op.bytes) != cudaSuccess) {
        cudaGetLastError();
        op.dev = nullptr;
        return op;
    }
    cudaMemcpy(op.dev, P.data(), op.bytes, cudaMemcpyHostToDevice);
    return op;
}

void translate_free(TranslateOp& op) {
    if (op.dev) cudaFree(op.dev);
    op.dev = nullptr;
}

void translate_configure() {
    cudaFuncSetAttribute(k_translate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
}

// C[p * ldc + m] (=|+=) sum_k W[m][k] X[p * ldx + k] for boxes p < N.  With ksplit > 1 and
// `work` (>= ksplit * N * ldc floats, ldc == Mtot) the K chunks are split over ksplit CTAs
// and the partial products summed in a fixed order.  wait_limit: the bound of the pipeline's
// waits in clock cycles, 0 for the default (about 2 s); lose_copies: the test hook above.
void translate_tc(const TranslateOp& op, const float* X, int ldx, int N, float* C, int ldc, bool accumulate,
                  int* status, cudaStream_t st, int ksplit, float* work, long long wait_limit, bool lose_copies) {
    if (N <= 0) return;
    const long long wlim = wait_limit > 0 ? wait_limit : kGWaitLimit;
    ksplit = std::max(1, std::min(ksplit, op.nkc));
    const bool split = ksplit > 1 && work && ldc == op.Mtot;
    const int kps = (op.nkc + (split ? ksplit : 1) - 1) / (split ? ksplit : 1);
    const int nz = (op.nkc + kps - 1) / kps;  // every slice has at least one chunk
    dim3 grid((N + kGBoxes - 1) / kGBoxes, op.nmt, nz);
    if (split) {
        const long cst = (long)N * ldc;
        k_translate_tc<<<grid, kGThreads, kGSmem, st>>>(op.dev, op.Mtot, op.nkc, op.K, X, ldx, N, work, ldc, 0, kps,
                                                        cst, status, wlim, lose_copies ? 1 : 0);
        const long tot = (long)N * ldc;
        k_translate_sum<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(N, ldc, nz, work, cst, C, accumulate ? 1 : 0);
    } else {
        k_translate_tc<<<grid, kGThreads, kGSmem, st>>>(op.dev, op.Mtot, op.nkc, op.K, X, ldx, N, C, ldc,
                                                        accumulate ? 1 : 0, kps, 0, status, wlim,
                                                        lose_copies ? 1 : 0);
    }
}

}  // namespace fmmcph
