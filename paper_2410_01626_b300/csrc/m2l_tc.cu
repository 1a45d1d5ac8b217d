// M2L on the 5th-generation tensor cores: tcgen05.mma kind::tf32, FP32 accumulation in TMEM.
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
// A CTA owns 256 consecutive "virtual rows" r0..r0+255 of the target class (interior rows
// are targets, ghost rows are discarded) and accumulates D[coef_out][row] in TMEM:
//   A = T_o chunk      (M = 128 output coefficients x K = 32 input coefficients), smem
//   B = source slab    (N = 256 rows x K = 32) -- one slab per (pi, K chunk) serves all
//                      deltas: the B descriptor just starts delta rows further in.
// Warp 0 lane 0 streams slabs and operator chunks with cp.async.bulk into a 3-stage ring;
// warp 1 lane 0 issues the MMAs; all four warps drain TMEM into the Morton-ordered L.
// Every wait is bounded; on expiry the CTA flags FMM_DEV_TIMEOUT and returns cleanly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmcph {

namespace {

constexpr int kTcRows = 256;    // virtual rows (N) per CTA
constexpr int kTcStages = 3;    // operator-chunk ring depth
constexpr int kTcChunk = 32;    // input coefficients per K chunk (4 MMAs of K = 8)
constexpr int kTcKG = kTcChunk / 4;
constexpr uint32_t kTcTBytes = 128 * kTcChunk * 4;  // one operator chunk: 128 x 32 fp32
constexpr long long kWaitLimit = 4000000000LL;    // clock cycles (about 2 s)

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

// Pack one level's multipoles into [class][kgroup][(n+2)^3 rows][4], rounded to TF32
// (round to nearest: the tensor core itself would truncate).
__global__ void k_m2l_pack(int n, int R, int NKG, int ncp, int periodic, const float* __restrict__ Mlev,
                           float* __restrict__ Mtc) {
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = 8L * NKG * R;
    if (tid >= total) return;
    const int row = (int)(tid % R);
    const int g = (int)((tid / R) % NKG);
    const int cls = (int)(tid / ((long)R * NKG));
    const int m2 = n + 2;
    int i = row / (m2 * m2) - 1, j = (row / m2) % m2 - 1, k = row % m2 - 1;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = 4 * g < ncp;
    if (periodic) {
        i = (i + n) % n;
        j = (j + n) % n;
        k = (k + n) % n;
    } else {
        ok = ok && i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n;
    }
    if (ok) {
        const uint32_t box = ((spread3_tc(i) | (spread3_tc(j) << 1) | (spread3_tc(k) << 2)) << 3) | (uint32_t)cls;
        v = *reinterpret_cast<const float4*>(Mlev + (long)box * ncp + 4 * g);
        v.x = tc::round_tf32(v.x);
        v.y = tc::round_tf32(v.y);
        v.z = tc::round_tf32(v.z);
        v.w = tc::round_tf32(v.w);
    }
    reinterpret_cast<float4*>(Mtc)[tid] = v;
}

struct TcTile {
    int level, cls, r0, pad;
};

__global__ void __launch_bounds__(128, 1)
    k_m2l_tc(const TcTile* __restrict__ tiles, TcLevels lv, const float* __restrict__ Mtc,
             const float* __restrict__ Ttc, float* __restrict__ L, int ncp, int NKC, int slab_rows,
             int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* slab = smem;
    uint8_t* tring = smem + (size_t)slab_rows * kTcKG * 16;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tring + (size_t)kTcStages * kTcTBytes);
    uint64_t* slab_full = bars + 0;
    uint64_t* slab_empty = bars + 1;
    uint64_t* done = bars + 2;
    uint64_t* t_full = bars + 3;
    uint64_t* t_empty = bars + 3 + kTcStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 + 2 * kTcStages);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const TcTile tile = tiles[blockIdx.x];
    const int lev = tile.level, c = tile.cls, r0 = tile.r0;
    const int n = lv.n[lev], R = lv.R[lev], S = lv.S[lev];
    const int m2 = n + 2;
    const int NKG = NKC * kTcKG;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;

    if (threadIdx.x == 0) {
        tc::mbar_init(slab_full, 1);
        tc::mbar_init(slab_empty, 1);
        tc::mbar_init(done, 1);
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(t_full + s, 1);
            tc::mbar_init(t_empty + s, 1);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kTcRows);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int slab_row0 = r0 - S;  // >= 0 by construction of the tile list
    const int rows_load = min(slab_rows, R - slab_row0);
    const float* Mlev = Mtc + lv.mtc_off[lev];

    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int it = 0, tcount = 0;
        bool ok = true;
        for (int pi = 0; pi < 8 && ok; ++pi) {
            const int px = pi & 1, py = (pi >> 1) & 1, pz = (pi >> 2) & 1;
            for (int ch = 0; ch < NKC && ok; ++ch) {
                if (it > 0 && !tc::mbar_wait(slab_empty, (it - 1) & 1, kWaitLimit)) {
                    ok = false;
                    break;
                }
                tc::mbar_arrive_expect_tx(slab_full, (uint32_t)rows_load * 16u * kTcKG);
                for (int g = 0; g < kTcKG; ++g) {
                    const float* src = Mlev + (((long)pi * NKG + ch * kTcKG + g) * R + slab_row0) * 4;
                    tc::bulk_g2s(slab + (size_t)g * slab_rows * 16, src, (uint32_t)rows_load * 16u, slab_full);
                }
                ++it;
                for (int d = 0; d < 27 && ok; ++d) {
                    const int dx = d / 9 - 1, dy = (d / 3) % 3 - 1, dz = d % 3 - 1;
                    const int ox = 2 * dx + px - cx, oy = 2 * dy + py - cy, oz = 2 * dz + pz - cz;
                    if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
                    const int s = tcount % kTcStages, u = tcount / kTcStages;
                    if (u > 0 && !tc::mbar_wait(t_empty + s, (u - 1) & 1, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    const int op = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
                    tc::mbar_arrive_expect_tx(t_full + s, kTcTBytes);
                    tc::bulk_g2s(tring + (size_t)s * kTcTBytes, Ttc + ((long)op * NKC + ch) * (kTcTBytes / 4),
                                 kTcTBytes, t_full + s);
                    ++tcount;
                }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, FMM_DEV_TIMEOUT);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = tc::idesc_tf32(128, kTcRows);
        const uint32_t slab_a = tc::smem_u32(slab), ring_a = tc::smem_u32(tring);
        const uint32_t kg_stride = (uint32_t)slab_rows * 16u;
        int it = 0, tcount = 0;
        uint32_t acc = 0;
        bool ok = true;
        for (int pi = 0; pi < 8 && ok; ++pi) {
            const int px = pi & 1, py = (pi >> 1) & 1, pz = (pi >> 2) & 1;
            for (int ch = 0; ch < NKC && ok; ++ch) {
                if (!tc::mbar_wait(slab_full, it & 1, kWaitLimit) || *abort_flag) {
                    ok = false;
                    break;
                }
                ++it;
                tc::fence_after_sync();
                for (int d = 0; d < 27 && ok; ++d) {
                    const int dx = d / 9 - 1, dy = (d / 3) % 3 - 1, dz = d % 3 - 1;
                    const int ox = 2 * dx + px - cx, oy = 2 * dy + py - cy, oz = 2 * dz + pz - cz;
                    if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
                    const int s = tcount % kTcStages, u = tcount / kTcStages;
                    if (!tc::mbar_wait(t_full + s, u & 1, kWaitLimit) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int shift = dx * m2 * m2 + dy * m2 + dz;
                    const uint32_t b_row = (uint32_t)(S + shift) * 16u;
                    const uint32_t a_base = ring_a + (uint32_t)s * kTcTBytes;
#pragma unroll
                    for (int ks = 0; ks < kTcChunk / 8; ++ks) {
                        const uint64_t ad = tc::smem_desc_kmajor(a_base + ks * 2 * 2048u, 2048u, 128u);
                        const uint64_t bd = tc::smem_desc_kmajor(slab_a + ks * 2 * kg_stride + b_row, kg_stride, 128u);
                        tc::mma_tf32(tmem, ad, bd, idesc, acc);
                        acc = 1;
                    }
                    tc::mma_commit(t_empty + s);
                    ++tcount;
                }
                tc::mma_commit(slab_empty);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, FMM_DEV_TIMEOUT);
        }
        tc::mma_commit(done);  // arrives once every issued MMA has completed
    }
    __syncwarp();

    // ---------------- epilogue: TMEM -> L (Morton order) ----------------
    const bool done_ok = tc::mbar_wait(done, 0, kWaitLimit);
    tc::fence_after_sync();
    if (done_ok && !*abort_flag) {
        const int j = warp * 32 + lane;  // output coefficient = TMEM lane
        float* Ll = L + lv.l_off[lev] * (long)ncp;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < kTcRows; cb += 16) {
            float v[16];
            tc::tmem_ld16(taddr + cb, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int r = r0 + cb + q;
                if (r >= R) continue;
                const int ip = r / (m2 * m2), jp = (r / m2) % m2, kp = r % m2;
                if (ip < 1 || ip > n || jp < 1 || jp > n || kp < 1 || kp > n) continue;
                const uint32_t box =
                    ((spread3_tc(ip - 1) | (spread3_tc(jp - 1) << 1) | (spread3_tc(kp - 1) << 2)) << 3) | (uint32_t)c;
                if (j < ncp) Ll[(long)box * ncp + j] = v[q];
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, FMM_DEV_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kTcRows);
}

}  // namespace

// ------------------------------------------------------------------------------------------
struct TcState {
    float* Mtc = nullptr;
    float* Ttc = nullptr;
    TcTile* tiles = nullptr;
    int ntiles = 0;
    int NKC = 0;
    int slab_rows = 0;
    size_t smem = 0;
    TcLevels lv{};
    std::vector<long> pack_off;
};

bool m2l_tc_supported(const Handle* h) {
    // M = 128 output coefficients per MMA; the slab of the deepest level fits in shared memory
    return h->precision == FMM_MIXED_TF32 && h->ncp <= 128 && h->depth <= 5;
}

static TcState* tc_state(Handle* h) { return reinterpret_cast<TcState*>(h->tc); }

int m2l_tc_setup(Handle* h, const std::vector<float>& T_rowmajor /*[343][nc][nc] j-major*/) {
    TcState* st = new TcState();
    h->tc = st;
    const int nc = h->nc, ncp = h->ncp, d = h->depth;
    st->NKC = (ncp + kTcChunk - 1) / kTcChunk;
    const int NKG = st->NKC * kTcKG;
    // operator chunks [op][chunk][kgroup][j(128)][4], rounded to TF32 (nearest, ties away)
    std::vector<float> T((size_t)kNumOps * st->NKC * 128 * kTcChunk, 0.f);
    auto tf32 = [](float x) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        float y;
        std::memcpy(&y, &u, 4);
        return y;
    };
    for (int op = 0; op < kNumOps; ++op)
        for (int jj = 0; jj < nc; ++jj)
            for (int k = 0; k < nc; ++k) {
                const float v = T_rowmajor[((size_t)op * nc + jj) * nc + k];
                const int ch = k / kTcChunk, g = (k % kTcChunk) / 4, e = k % 4;
                T[((((size_t)op * st->NKC + ch) * kTcKG + g) * 128 + jj) * 4 + e] = tf32(v);
            }
    // packed multipole levels
    long off = 0;
    for (int l = 0; l <= kMaxDepth; ++l) {
        st->lv.n[l] = st->lv.R[l] = st->lv.S[l] = 0;
        st->lv.mtc_off[l] = 0;
        st->lv.l_off[l] = 0;
    }
    std::vector<TcTile> tiles;
    int max_S = 0;
    for (int l = h->lmin; l <= d; ++l) {
        const int n = 1 << (l - 1);
        const int R = (n + 2) * (n + 2) * (n + 2);
        const int S = dmax_shift(n);
        st->lv.n[l] = n;
        st->lv.R[l] = R;
        st->lv.S[l] = S;
        st->lv.mtc_off[l] = off;
        st->lv.l_off[l] = h->lvl_off[l];
        off += 8L * NKG * R * 4;
        max_S = std::max(max_S, S);
        for (int c = 0; c < 8; ++c)
            for (int r0 = S; r0 < R - S; r0 += kTcRows) tiles.push_back({l, c, r0, 0});
    }
    st->slab_rows = kTcRows + 2 * max_S;
    st->smem = (size_t)st->slab_rows * kTcKG * 16 + (size_t)kTcStages * kTcTBytes + 256;
    st->ntiles = (int)tiles.size();
    if (cudaMalloc(&st->Ttc, sizeof(float) * T.size()) != cudaSuccess ||
        cudaMalloc(&st->Mtc, sizeof(float) * (off > 0 ? off : 4)) != cudaSuccess ||
        cudaMalloc(&st->tiles, sizeof(TcTile) * (tiles.empty() ? 1 : tiles.size())) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ERR_OOM;
    }
    cudaMemcpy(st->Ttc, T.data(), sizeof(float) * T.size(), cudaMemcpyHostToDevice);
    if (!tiles.empty()) cudaMemcpy(st->tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice);
    if (st->smem > 227 * 1024) return FMM_ERR_ARG;
    cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem);
    return FMM_OK;
}

void m2l_tc_free(Handle* h) {
    TcState* st = tc_state(h);
    if (!st) return;
    if (st->Mtc) cudaFree(st->Mtc);
    if (st->Ttc) cudaFree(st->Ttc);
    if (st->tiles) cudaFree(st->tiles);
    delete st;
    h->tc = nullptr;
}

int m2l_tc_launches(const Handle* h) {
    return (h->depth - h->lmin + 1) + 1;  // one pack per level + the MMA kernel
}

void launch_m2l_tc(Handle* h, cudaStream_t stream) {
    TcState* st = tc_state(h);
    const int NKG = st->NKC * kTcKG;
    for (int l = h->lmin; l <= h->depth; ++l) {
        const long total = 8L * NKG * st->lv.R[l];
        k_m2l_pack<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
            st->lv.n[l], st->lv.R[l], NKG, h->ncp, h->periodic, h->M + h->lvl_off[l] * h->ncp,
            st->Mtc + st->lv.mtc_off[l]);
    }
    if (st->ntiles > 0)
        k_m2l_tc<<<st->ntiles, 128, st->smem, stream>>>(st->tiles, st->lv, st->Mtc, st->Ttc, h->L, h->ncp, st->NKC,
                                                         st->slab_rows, h->status);
}

}  // namespace fmmcph
