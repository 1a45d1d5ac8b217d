// CUDA kernels of one FMM evaluation (sm_103a).
//
// Stages (launch_eval at the end of this file places them on the caller's stream and on the
// handle's chain and side streams):
//   binning   k_bin_count -> k_bin_scan -> k_bin_place -> k_bin_order_gather (counting sort by leaf)
//             (Morton keys of the leaf cells, stable on (key, index); the gather also forms
//             q_i = qA_i + lambda_s (qB_i - qA_i), Sec. 2.1 Eq. 1 with charge-only forms)
//   P2M       k_p2m<P>        16 leaves per block, two column sets x four atom slices per leaf, sums in registers
//   M2M       k_translate_tc  per level, one product over the 8 contiguous children (translate_tc.cu;
//                             FP32 SGEMM in the FP32 mode)
//   root      k_qdt, k_root, k_lattice (periodic) FP64 root multipole, lattice operator, Q/D/T
//   M2L       k_m2l_fp32 (FP32 CUDA cores) or the tcgen05 kernel in m2l_tc.cu
//   L2L       k_translate_tc  per level, one product into the 8 contiguous children (as M2M)
//   outputs   k_far_out<P>    far field per atom (L2P + periodic background term) + near field -> F, phi, E partials
//             k_p2p           P2P over the 27 neighbour leaves + forces / potential / energy
//   final     k_final         E (FP64, fixed-order reduction) and dV/dlambda per site
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "bounds.cuh"
#include "fmm_internal.h"
#include "sgemm.cuh"
#include "tc_ptx.cuh"

namespace fmmcph {

FMM_BC_TAKE(bc_take_kernels)

// ---- constant tables of the normalised regular-harmonic recurrences ----
__constant__ float c_dg[kMaxP + 2];                   // sqrt((2m-1)/(2m))
__constant__ float c_ra[kMaxP + 2][kMaxP + 2];        // (2n-1)/sqrt((n+m)(n-m))
__constant__ float c_rb[kMaxP + 2][kMaxP + 2];        // sqrt((n+m-1)(n-m-1)/((n+m)(n-m)))
__constant__ float c_g1[kMaxP + 2][kMaxP + 2];        // sqrt((n+m+1)(n+m+2))
__constant__ float c_g2[kMaxP + 2][kMaxP + 2];        // sqrt((n-m+1)(n-m+2))
__constant__ float c_g3[kMaxP + 2][kMaxP + 2];        // sqrt((n+1+m)(n+1-m))

void upload_constants(int /*p*/) {
    float dg[kMaxP + 2] = {0};
    static float ra[kMaxP + 2][kMaxP + 2], rb[kMaxP + 2][kMaxP + 2], g1[kMaxP + 2][kMaxP + 2],
        g2[kMaxP + 2][kMaxP + 2], g3[kMaxP + 2][kMaxP + 2];
    for (int m = 1; m < kMaxP + 2; ++m) dg[m] = (float)std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    for (int n = 0; n < kMaxP + 2; ++n)
        for (int m = 0; m < kMaxP + 2; ++m) {
            ra[n][m] = rb[n][m] = 0.f;
            if (n > m) {
                ra[n][m] = (float)((2.0 * n - 1.0) / std::sqrt(double(n + m) * (n - m)));
                if (n >= m + 2)
                    rb[n][m] = (float)std::sqrt(double(n + m - 1) * (n - m - 1) / (double(n + m) * (n - m)));
            }
            g1[n][m] = (float)std::sqrt(double(n + m + 1) * (n + m + 2));
            g2[n][m] = (n >= m) ? (float)std::sqrt(double(n - m + 1) * (n - m + 2)) : 0.f;
            g3[n][m] = (n + 1 >= m) ? (float)std::sqrt(double(n + 1 + m) * (n + 1 - m)) : 0.f;
        }
    cudaMemcpyToSymbol(c_dg, dg, sizeof(dg));
    cudaMemcpyToSymbol(c_ra, ra, sizeof(ra));
    cudaMemcpyToSymbol(c_rb, rb, sizeof(rb));
    cudaMemcpyToSymbol(c_g1, g1, sizeof(g1));
    cudaMemcpyToSymbol(c_g2, g2, sizeof(g2));
    cudaMemcpyToSymbol(c_g3, g3, sizeof(g3));
}

// ---- Morton helpers (up to 10 bits per axis) ----
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030C30C3u;
    v = (v ^ (v >> 4)) & 0x0300F00Fu;
    v = (v ^ (v >> 8)) & 0x030000FFu;
    v = (v ^ (v >> 16)) & 0x000003FFu;
    return v;
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

struct BoxGeom {
    double o0, o1, o2, L, s;
    int nb, depth, periodic;
};

// Wrapped (periodic) or raw (open) coordinate relative to the origin, exactly
// as the binning specification states it (FP64, no FMA contraction).
__device__ __forceinline__ double wrap_coord(double x, double o, double L, int periodic) {
    double u = __dsub_rn(x, o);
    if (periodic && !(u >= 0.0 && u < L)) {  // inside [0, L) the formula leaves u unchanged
        u = __dsub_rn(u, __dmul_rn(L, floor(__ddiv_rn(u, L))));
        if (u < 0.0 || u >= L) u = 0.0;
    }
    return u;
}

__device__ __forceinline__ int cell_of(double u, double s, int nb) {
    double f = floor(__dmul_rn(u, s));
    if (!(f >= 0.0)) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (int)f;
}

// Leaf cell of one coordinate, bit-identical to the FP64 specification above.  FP32 first:
// with of = fl32(o), sf = fl32(s), u32 = fl32(x - of), t32 = fl32(u32 sf),
//   |u32 - (x - o)| <= 2^-24 (|o| + |x - of|)                    <= E_u = 2^-23 (|x| + 2|o|),
//   |t32 - (x - o) s| <= 2^-24 |u32| (sf + s) + s E_u            <= E_t = s (2^-22 |u32| + E_u),
// and the FP64 value differs from (x - o) s by far less than E_t.  When u32 is more than E_u
// (plus the rounding of L) inside (0, L) -- so FP64 neither wraps nor flags the domain -- and
// t32 is more than E_t from both integers around it, floor(t32) is the FP64 cell; otherwise
// the FP64 arithmetic decides.  *bad is set for an open-box coordinate outside [0, L].
__device__ __forceinline__ int cell_fast(float xf, double o, float of, BoxGeom g, float Lf, float sf, bool& bad) {
    const float u32 = xf - of;
    const float eu = 1.1920929e-7f * (fabsf(xf) + 2.f * fabsf(of)) + 1e-30f;  // 2^-23 (|x| + 2|o|)
    if (u32 > eu && u32 < Lf - eu - 1.1920929e-7f * Lf) {
        const float t32 = u32 * sf;
        const float et = sf * (2.3841858e-7f * u32 + eu) * 1.0001f;             // 2^-22 |u32| + E_u
        const float c = floorf(t32);
        if (t32 - c > et && c + 1.f - t32 > et) return min((int)c, g.nb - 1);
    }
    const double u = wrap_coord((double)xf, o, g.L, g.periodic);
    if (!g.periodic && !(u >= 0.0 && u <= g.L)) bad = true;
    return cell_of(u, g.s, g.nb);
}

__device__ __forceinline__ uint32_t leaf_key(const float* __restrict__ x, int i, const BoxGeom& g, bool& bad) {
    const float Lf = (float)g.L, sf = (float)g.s;
    const int cx = cell_fast(x[3 * i], g.o0, (float)g.o0, g, Lf, sf, bad);
    const int cy = cell_fast(x[3 * i + 1], g.o1, (float)g.o1, g, Lf, sf, bad);
    const int cz = cell_fast(x[3 * i + 2], g.o2, (float)g.o2, g, Lf, sf, bad);
    return morton3(cx, cy, cz);
}

__global__ void k_keys(int n, const float* __restrict__ x, BoxGeom g, uint32_t* __restrict__ key,
                       uint32_t* __restrict__ val, int* __restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool bad = false;
    key[i] = leaf_key(x, i, g, bad);
    val[i] = (uint32_t)i;
    if (bad && status) atomicOr(status, FMM_DEV_DOMAIN);
}

// ---- binning as a counting sort by leaf ----
// (1) k_bin_count: key of every atom and a claim on a slot of its leaf (atomic, so the slot
//     order inside a leaf is arbitrary), and the atom counts of tiles of kScanTile leaves
//     (a block histogram in shared memory, then one atomic per tile and block); (2) k_bin_scan,
//     one block per tile: the tile's offset is the sum of the tile counts before it, then an
//     exclusive scan of its leaf counts -> start, count (and the counters are cleared for the
//     next call); (3) k_bin_place: atom i goes to start[key] + slot, and the tile counts are
//     cleared; (4) k_bin_order_gather: a warp takes two leaves (a half-warp each when both hold at most
//     16 atoms, else one after the other) and puts each leaf's atoms in ascending
//     input index -- exactly the order of a stable sort on (key, index) -- and gathers positions
//     and charges in that order.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;                          // leaf counts per thread, vector loads
constexpr int kScanTile = kScanThreads * kScanPer;    // leaves per scan block
constexpr int kMaxScanTiles = (1 << (3 * kMaxDepth)) / kScanTile;
constexpr int kCountThreads = 256;

inline int scan_tiles(int nleaf) { return (nleaf + kScanTile - 1) / kScanTile; }
int leafcnt_words(int nleaf) { return nleaf + scan_tiles(nleaf); }

__global__ void __launch_bounds__(kCountThreads) k_bin_count(int n, const float* __restrict__ x, BoxGeom g,
                                                             uint32_t* __restrict__ key, uint32_t* __restrict__ slot,
                                                             uint32_t* __restrict__ leafcnt, int ntiles,
                                                             uint32_t* __restrict__ tilecnt,
                                                             int* __restrict__ status, int2* __restrict__ items) {
    __shared__ uint32_t hist[kMaxScanTiles];
    if (items && blockIdx.x == 0 && threadIdx.x == 0) items[0].x = 0;  // the near field's item list (k_bin_order_gather)
    for (int t = threadIdx.x; t < ntiles; t += kCountThreads) hist[t] = 0u;
    __syncthreads();
    const int i = blockIdx.x * kCountThreads + threadIdx.x;
    if (i < n) {
        bool bad = false;
        const uint32_t k = leaf_key(x, i, g, bad);
        key[i] = k;
        if (FMM_IN(k, 1u << (3 * g.depth))) {
            slot[i] = atomicAdd(leafcnt + k, 1u);
            if (ntiles > 1) atomicAdd(hist + k / kScanTile, 1u);
        }
        if (bad) atomicOr(status, FMM_DEV_DOMAIN);
    }
    if (ntiles > 1) {
        __syncthreads();
        for (int t = threadIdx.x; t < ntiles; t += kCountThreads)
            if (hist[t]) atomicAdd(tilecnt + t, hist[t]);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_bin_scan(int nleaf, uint32_t* __restrict__ leafcnt,
                                                           const uint32_t* __restrict__ tilecnt,
                                                           uint32_t* __restrict__ start, uint32_t* __restrict__ count) {
    __shared__ uint32_t wsum[kScanThreads / 32];
    __shared__ uint32_t wpre[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, b = blockIdx.x;
    // the leaves before this tile: the sum of the tile counts before it (integers: any order)
    uint32_t pre = 0;
    for (int i = t; i < b; i += kScanThreads) pre += tilecnt[i];
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, k);
    if (lane == 0) wpre[w] = pre;
    const int l0 = b * kScanTile + kScanPer * t;
    const bool whole = l0 + kScanPer <= nleaf;  // l0 is a multiple of 16: aligned vector access
    uint32_t v[kScanPer], tot = 0;
    if (whole) {
#pragma unroll
        for (int e = 0; e < kScanPer; e += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(leafcnt + l0 + e);
            v[e] = q.x, v[e + 1] = q.y, v[e + 2] = q.z, v[e + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) v[e] = l0 + e < nleaf ? leafcnt[l0 + e] : 0u;
    }
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) tot += v[e];
    uint32_t x = tot;  // inclusive scan of the thread totals
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
        if (lane >= k) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t base = 0;
#pragma unroll
    for (int j = 0; j < kScanThreads / 32; ++j) {
        base += wpre[j];
        if (j < w) base += wsum[j];
    }
    uint32_t run = base + x - tot;
    uint32_t st[kScanPer];
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        st[e] = run;
        run += v[e];
    }
    if (whole) {
#pragma unroll
        for (int e = 0; e < kScanPer; e += 4) {
            *reinterpret_cast<uint4*>(start + l0 + e) = make_uint4(st[e], st[e + 1], st[e + 2], st[e + 3]);
            *reinterpret_cast<uint4*>(count + l0 + e) = make_uint4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            *reinterpret_cast<uint4*>(leafcnt + l0 + e) = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
#pragma unroll
        for (int e = 0; e < kScanPer; ++e) {
            if (l0 + e < nleaf) {
                start[l0 + e] = st[e];
                count[l0 + e] = v[e];
                leafcnt[l0 + e] = 0u;
            }
        }
    }
}

__global__ void k_bin_place(int n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ slot,
                            const uint32_t* __restrict__ start, uint32_t* __restrict__ placed, int ntiles,
                            uint32_t* __restrict__ tilecnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0)  // every k_bin_scan block has read them
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) tilecnt[t] = 0u;
    if (i >= n) return;
    const uint32_t d = start[key[i]] + slot[i];
    if (FMM_IN(d, n)) placed[d] = (uint32_t)i;
}

// The charge forms of the atoms and the site coordinates (Sec. 2.1, Eq. 1 and Eq. 2).
struct ChargeForms {
    const float* q[4];     // forms A, B (two-form sites), + C, D (four-form sites)
    int nforms;            // 2: q = qA + lambda (qB - qA); 4: bilinear in (lambda_p, lambda_t)
    const int32_t* site;
    int K;
    const float* lam;      // [K] or [2K] = (lambda_p, lambda_t) per site
    float* dq;             // dq/dlambda (two forms) or dq/dlambda_p (four forms), sorted order
    float* dqt;            // dq/dlambda_t (four forms), sorted order
};

// Position and charges of input atom i at sorted slot s (the gather of the binning step).
__device__ __forceinline__ void gather_atom(int i, int s, const float* __restrict__ x, const BoxGeom& g,
                                            const ChargeForms& cf, float4* __restrict__ pos,
                                            uint32_t* __restrict__ inv, int* __restrict__ status) {
    float u[3];
    const double o[3] = {g.o0, g.o1, g.o2};
    const float Lf = (float)g.L;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xf = x[3 * i + a], of = (float)o[a];
        const float u32 = xf - of;
        const float eu = 1.1920929e-7f * (fabsf(xf) + 2.f * fabsf(of)) + 1e-30f;
        if (g.periodic && !(u32 > eu && u32 < Lf - eu - 1.1920929e-7f * Lf))
            u[a] = (float)wrap_coord((double)xf, o[a], g.L, 1);
        else
            u[a] = u32;
    }
    const float a = cf.q[0][i];
    const int st = cf.site[i];
    float d = 0.f, dt = 0.f, q = a;
    if (st >= 0) {
        if (st < cf.K) {
            if (cf.nforms == 4) {
                const float lp = cf.lam[2 * st], lt = cf.lam[2 * st + 1];
                const float b = cf.q[1][i], c = cf.q[2][i], e = cf.q[3][i];
                const float ab = fmaf(lt, b - a, a), cd = fmaf(lt, e - c, c);
                q = fmaf(lp, cd - ab, ab);
                d = cd - ab;
                dt = fmaf(lp, (e - c) - (b - a), b - a);
            } else {
                const float b = cf.q[1][i];
                d = b - a;
                q = fmaf(cf.lam[st], d, a);
            }
        } else {
            atomicOr(status, FMM_DEV_SITE);
        }
    }
    pos[s] = make_float4(u[0], u[1], u[2], q);
    cf.dq[s] = d;
    if (cf.nforms == 4) cf.dqt[s] = dt;
    inv[i] = (uint32_t)s;
}

// The near field takes leaves with more than kNearTile atoms in tiles of kNearTile targets, listed
// by the binning (k_bin_order_gather) as items (leaf, tile) after a count in items[0].x.
constexpr int kNearTile = 64;

__global__ void __launch_bounds__(128) k_bin_order_gather(int nleaf, const uint32_t* __restrict__ start,
                                                          const uint32_t* __restrict__ count,
                                                          const uint32_t* __restrict__ placed,
                                                          uint32_t* __restrict__ perm, uint32_t* __restrict__ skey,
                                                          const float* __restrict__ x, BoxGeom g, ChargeForms cf,
                                                          float4* __restrict__ pos, uint32_t* __restrict__ inv,
                                                          int* __restrict__ status, int2* __restrict__ items,
                                                          int items_cap, int n) {
    // a warp takes leaves l0 and l0 + 1
    const int l0 = 2 * (blockIdx.x * 4 + (threadIdx.x >> 5)), lane = threadIdx.x & 31;
    if (l0 >= nleaf) return;
    const bool two = l0 + 1 < nleaf;
    const int c0 = (int)count[l0], c1 = two ? (int)count[l0 + 1] : 0;
    if (lane == 0 && items) {  // the near field's work items of leaves above kNearTile atoms
        for (int q = 0; q < (two ? 2 : 1); ++q) {
            const int c = q ? c1 : c0;
            if (c <= kNearTile) continue;
            const int nt = (c + kNearTile - 1) / kNearTile;
            const int base = atomicAdd(&items[0].x, nt);
            for (int t = 0; t < nt && base + t < items_cap; ++t) items[1 + base + t] = make_int2(l0 + q, t);
        }
    }
    if (c0 <= 16 && c1 <= 16) {  // one leaf per half-warp, one atom per lane
        const int half = lane >> 4, sub = lane & 15, c = half ? c1 : c0;
        const int leaf = l0 + half;
        const int st = c > 0 ? (int)start[leaf] : 0;
        const uint32_t v = sub < c && FMM_IN(st + sub, n) ? placed[st + sub] : 0xFFFFFFFFu;
        int r = 0;  // rank = number of smaller indices in the leaf (padding is never smaller)
        for (int k = 0; k < 16; ++k) r += __shfl_sync(0xffffffffu, v, k, 16) < v ? 1 : 0;
        if (sub < c && FMM_IN(v, n) && FMM_IN(st + r, n)) {
            perm[st + r] = v;
            skey[st + r] = (uint32_t)leaf;
            gather_atom((int)v, st + r, x, g, cf, pos, inv, status);
        }
        return;
    }
    for (int leaf = l0; leaf < l0 + (two ? 2 : 1); ++leaf) {
        const int st = (int)start[leaf], c = leaf == l0 ? c0 : c1;
        if (!FMM_OK(st >= 0 && st + c <= n)) continue;  // (st and c are the warp's own: no divergence)
        if (c <= 32) {  // the whole leaf in one register per lane
            const uint32_t v = lane < c ? placed[st + lane] : 0xFFFFFFFFu;
            int r = 0;
            for (int k = 0; k < c; ++k) r += __shfl_sync(0xffffffffu, v, k) < v ? 1 : 0;
            if (lane < c && FMM_IN(v, n)) {
                perm[st + r] = v;
                skey[st + r] = (uint32_t)leaf;
                gather_atom((int)v, st + r, x, g, cf, pos, inv, status);
            }
            continue;
        }
        // larger leaves: the same ranks by a pass over the leaf per element (O(c^2 / 32) per warp,
        // the order of the leaf's own near-field work)
        for (int e = lane; e < c; e += 32) {
            const uint32_t v = placed[st + e];
            int r = 0;
            for (int k = 0; k < c; ++k) r += placed[st + k] < v ? 1 : 0;
            if (!FMM_IN(v, n)) continue;
            perm[st + r] = v;
            skey[st + r] = (uint32_t)leaf;
            gather_atom((int)v, st + r, x, g, cf, pos, inv, status);
        }
    }
}

// ---- stable LSD radix sort, 8-bit digits ----
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortSub = 512;  // keys per warp sub-chunk
constexpr int kSortTile = kSortWarps * kSortSub;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(int n, const uint32_t* __restrict__ keys,
                                                            int shift, uint32_t* __restrict__ table,
                                                            int nblk) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int j = threadIdx.x; j < kSortTile; j += kSortThreads) {
        int i = base + j;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    table[threadIdx.x * nblk + blockIdx.x] = hist[threadIdx.x];
}

// exclusive scan of the digit-major table [256 digits][nblk], one block of 1024 threads:
// each warp scans whole digit rows with coalesced loads, then the 256 digit totals are scanned
// and added back.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ table, int total) {
    __shared__ uint32_t dtot[256];
    __shared__ uint32_t wsum[32];
    const int nblk = total / 256;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = w; d < 256; d += 32) {  // row d: exclusive scan within the row
        uint32_t carry = 0;
        for (int b0 = 0; b0 < nblk; b0 += 32) {
            const int b = b0 + lane;
            const uint32_t v = (b < nblk) ? table[d * nblk + b] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
                if (lane >= k) x += y;
            }
            if (b < nblk) table[d * nblk + b] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) dtot[d] = carry;
    }
    __syncthreads();
    // exclusive scan of the 256 digit totals (threads 0..255)
    uint32_t v = (threadIdx.x < 256) ? dtot[threadIdx.x] : 0u, x = v;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
        if (lane >= k) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t z = (lane < 8) ? wsum[lane] : 0u;
#pragma unroll
        for (int k = 1; k < 8; k <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, k);
            if (lane >= k) z += y;
        }
        if (lane < 8) wsum[lane] = z;
    }
    __syncthreads();
    if (threadIdx.x < 256) dtot[threadIdx.x] = x - v + (w > 0 ? wsum[w - 1] : 0u);
    __syncthreads();
    for (int e = threadIdx.x; e < total; e += 1024) table[e] += dtot[e / nblk];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(int n, const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, int shift,
                                                               const uint32_t* __restrict__ table,
                                                               int nblk) {
    __shared__ uint32_t woff[kSortWarps][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&woff[0][0])[d] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile + w * kSortSub;
    for (int j = lane; j < kSortSub; j += 32) {
        int i = base + j;
        if (i < n) atomicAdd(&woff[w][(kin[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // 256 threads = 256 digits
        uint32_t run = table[d * nblk + blockIdx.x];
        for (int ww = 0; ww < kSortWarps; ++ww) {
            uint32_t c = woff[ww][d];
            woff[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (int g = 0; g < kSortSub; g += 32) {
        int i = base + g + lane;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u;
        uint32_t digit = valid ? ((k >> shift) & 255u) : (256u + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, digit);
        uint32_t rank = __popc(peers & lt);
        if (valid) {
            uint32_t pos = woff[w][digit] + rank;
            kout[pos] = k;
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) woff[w][digit] += __popc(peers);
        __syncwarp();
    }
}

// leaf ranges by binary search over the sorted keys (empty leaves start at their insertion point)
__global__ void k_ranges(int n, int nleaf, const uint32_t* __restrict__ skey, uint32_t* __restrict__ start,
                         uint32_t* __restrict__ count) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    auto lower = [&](uint32_t v) {
        int lo = 0, hi = n;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (skey[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    int s = lower((uint32_t)b), e = lower((uint32_t)b + 1u);
    start[b] = (uint32_t)s;
    count[b] = (uint32_t)(e - s);
}

// ---- normalised regular solid harmonics, real form ----
// R_hat_n^m(u) for n = 0..P, m = 0..n via the column recurrences; `visit(n, m, re, im)`.
template <int P, class F>
__device__ __forceinline__ void regular_harmonics(float x, float y, float z, F&& visit) {
    const float rho2 = x * x + y * y + z * z;
    float dr = 1.f, di = 0.f;
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        if (m > 0) {
            const float t = (dr * x + di * y) * c_dg[m];
            di = (di * x - dr * y) * c_dg[m];
            dr = t;
        }
        float pr = dr, pi = di, ppr = 0.f, ppi = 0.f;
#pragma unroll
        for (int n = m; n <= P; ++n) {
            if (n > m) {
                const float a = c_ra[n][m] * z, b = c_rb[n][m] * rho2;
                const float nr = a * pr - b * ppr, ni = a * pi - b * ppi;
                ppr = pr;
                ppi = pi;
                pr = nr;
                pi = ni;
            }
            visit(n, m, pr, pi);
        }
    }
}

// Columns m in [M0, M1] only (the m = 0 .. M1 diagonal chain is still walked).
template <int P, int M0, int M1, class F>
__device__ __forceinline__ void regular_harmonics_cols(float x, float y, float z, F&& visit) {
    const float rho2 = x * x + y * y + z * z;
    float dr = 1.f, di = 0.f;
#pragma unroll
    for (int m = 0; m <= M1; ++m) {
        if (m > 0) {
            const float t = (dr * x + di * y) * c_dg[m];
            di = (di * x - dr * y) * c_dg[m];
            dr = t;
        }
        if (m < M0) continue;
        float pr = dr, pi = di, ppr = 0.f, ppi = 0.f;
#pragma unroll
        for (int n = m; n <= P; ++n) {
            if (n > m) {
                const float a = c_ra[n][m] * z, b = c_rb[n][m] * rho2;
                const float nr = a * pr - b * ppr, ni = a * pi - b * ppi;
                ppr = pr;
                ppi = pi;
                pr = nr;
                pi = ni;
            }
            visit(n, m, pr, pi);
        }
    }
}

// P2M: M_b = sum over the leaf's atoms of q R_hat_n^m(u), u = (x - c_b) / h, with the
// normalised regular harmonics of the recurrence above, every sum in registers.  A block takes
// 32 leaves: warps 0-1 the columns m < MS and warps 2-3 the columns m >= MS of the recurrence
// (warp-uniform, so the two column sets never diverge in a warp; MS balances their cost, the
// diagonal chain to MS - 1 included).  Within a warp, lanes 2k and 2k+1 share leaf k of the
// warp's 16: lane 2k sums over the leaf's even atoms and lane 2k+1 over its odd atoms, each in
// order; one shuffle adds the two (a + b: the same value in both lanes), and the two lanes
// write alternate coefficients.  With no shared memory, 20 warps per SM are resident at p = 10.
// The warps of the columns m >= MS also sum the leaf's moments for the periodic correction,
// about the leaf centre: q_hi, q_lo (q_hi = q rounded to a multiple of 2^-11, so the FP32 sum
// of q_hi is exact and Q = sum q_hi + sum q_lo is good to FP64 level), q dx, q dy, q dz,
// q |d|^2.  k_qdt turns them into Q, D, T about the box centre in FP64 with all lanes busy:
// this GPU's FP64 pipe is narrow, so no FP64 instruction runs per atom or per leaf thread.
// Every sum runs in a fixed order, so the result is deterministic.
constexpr int kMom = 6;        // leaf moments for the periodic correction
constexpr int kMomStride = kLeafMomStride;  // floats per leaf in the moment array
template <int P>
struct P2mCfg {
    static constexpr int NC = (P + 1) * (P + 1);
    // column split: sum over m < MS of (P - m + 1), plus the chain to MS - 1, against the rest
    static constexpr int split() {
        int best = 1, bestd = 1 << 30;
        for (int ms = 1; ms <= P; ++ms) {
            int a = ms - 1, b = P;
            for (int m = 0; m <= P; ++m) (m < ms ? a : b) += P - m + 1;
            const int d = a > b ? a - b : b - a;
            if (d < bestd) {
                bestd = d;
                best = ms;
            }
        }
        return best;
    }
    static constexpr int MS = P >= 1 ? split() : 1;
};

constexpr int kP2mSlices = 4;   // lanes per leaf and column set, each taking every 4th atom
constexpr int kP2mLeaves = 64 / kP2mSlices;  // leaves per block of 4 warps (2 column sets)
template <int P, int M0, int M1, class F>
__device__ __forceinline__ void for_cols(F&& f) {  // the coefficient slots of columns M0 .. M1
#pragma unroll
    for (int m = M0; m <= M1; ++m)
#pragma unroll
        for (int n = m; n <= P; ++n) {
            if (m == 0) {
                f(n * n);
            } else {
                f(n * n + 2 * m - 1);
                f(n * n + 2 * m);
            }
        }
}
template <int P, int M0, int M1, bool MOM>
__device__ __forceinline__ void p2m_leaf_cols(const float4* __restrict__ pos, int st, int cnt, int par, float cx,
                                              float cy, float cz, float ih, float* acc, float* mom) {
    float4 nxt = par < cnt ? pos[st + par] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = par; k < cnt; k += kP2mSlices) {
        const float4 p4 = nxt;
        if (k + kP2mSlices < cnt) nxt = pos[st + k + kP2mSlices];  // the lane's next atom, in flight during this one
        const float q = p4.w, dx = p4.x - cx, dy = p4.y - cy, dz = p4.z - cz;
        regular_harmonics_cols<P, M0, M1>(dx * ih, dy * ih, dz * ih, [&](int n, int m, float re, float im) {
            if (m == 0) {
                acc[n * n] = fmaf(q, re, acc[n * n]);
            } else {
                acc[n * n + 2 * m - 1] = fmaf(q, re, acc[n * n + 2 * m - 1]);
                acc[n * n + 2 * m] = fmaf(-q, im, acc[n * n + 2 * m]);
            }
        });
        if (MOM) {
            const float qhi = rintf(q * 2048.f) * (1.f / 2048.f);
            mom[0] += qhi;
            mom[1] += q - qhi;
            mom[2] = fmaf(q, dx, mom[2]);
            mom[3] = fmaf(q, dy, mom[3]);
            mom[4] = fmaf(q, dz, mom[4]);
            mom[5] = fmaf(q, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), mom[5]);
        }
    }
#pragma unroll
    for (int d = 1; d < kP2mSlices; d <<= 1) {  // the leaf's slices, added in a fixed tree
#pragma unroll
        for (int i = 0; i < (MOM ? kMom : 0); ++i) mom[i] += __shfl_xor_sync(0xffffffffu, mom[i], d);
        for_cols<P, M0, M1>([&](int i) { acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], d); });
    }
}
template <int P>
__global__ void __launch_bounds__(128, P <= 10 ? 5 : 3) k_p2m(int nleaf, float h, const uint32_t* __restrict__ start,
                                             const uint32_t* __restrict__ count, const float4* __restrict__ pos,
                                             float* __restrict__ M, int ncp, float* __restrict__ leafmom, int n) {
    using Cfg = P2mCfg<P>;
    constexpr int NC = Cfg::NC, MS = Cfg::MS;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int leaf = blockIdx.x * kP2mLeaves + (w & 1) * (32 / kP2mSlices) + lane / kP2mSlices;
    const int par = lane % kP2mSlices;
    const bool valid = leaf < nleaf;
    const int st = valid ? (int)start[leaf] : 0;
    int cnt = valid ? (int)count[leaf] : 0;
    if (!FMM_OK(st >= 0 && st + cnt <= n)) cnt = 0;  // (the lanes still run the shuffles together)
    const uint32_t lf = valid ? (uint32_t)leaf : 0u;
    const float cx = (compact3(lf) + 0.5f) * h, cy = (compact3(lf >> 1) + 0.5f) * h,
                cz = (compact3(lf >> 2) + 0.5f) * h;
    const float ih = 1.0f / h;
    float acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.f;
    float mom[kMom];
#pragma unroll
    for (int i = 0; i < kMom; ++i) mom[i] = 0.f;
    float* out = M + (long)lf * ncp;
    auto put = [&](int i) {  // the lanes of a leaf write the slots in turn
        if (valid && i % kP2mSlices == par) out[i] = acc[i];
    };
    if (w < 2) {
        p2m_leaf_cols<P, 0, MS - 1, false>(pos, st, cnt, par, cx, cy, cz, ih, acc, mom);
        for_cols<P, 0, MS - 1>(put);
    } else {
        p2m_leaf_cols<P, MS, P, true>(pos, st, cnt, par, cx, cy, cz, ih, acc, mom);
        for_cols<P, MS, P>(put);
        if (valid) {
            for (int v = NC + par; v < ncp; v += kP2mSlices) out[v] = 0.f;
            if (leafmom && par == 0)
#pragma unroll
                for (int k = 0; k < kMom; ++k) leafmom[(long)lf * kMomStride + k] = mom[k];
        }
    }
}

// ---- periodic root: FP64 root multipole (M2M from level 1) and the Q, D, T sums ----
// Q = sum q, D = sum q u, T = sum q |u|^2 about the box centre, from the leaf moments about
// the leaf centres c (d = u - c):  D = sum q d + Q c,  T = sum q |d|^2 + 2 c . sum q d + Q |c|^2,
// in FP64, reduced in a fixed order: leaves -> kQdtBlocks partials (k_qdt) -> totals (k_lattice).
constexpr int kQdtBlocks = 64;
__global__ void __launch_bounds__(256) k_qdt(int nleaf, double h, double half_box, const float* __restrict__ leafmom,
                                             double* __restrict__ partial) {
    __shared__ double red[5][256];
    const int per = (nleaf + kQdtBlocks - 1) / kQdtBlocks;
    const int b0 = blockIdx.x * per, b1 = min(nleaf, b0 + per);
    double a[5] = {0, 0, 0, 0, 0};
    for (int l = b0 + threadIdx.x; l < b1; l += 256) {
        const float4 m0 = *reinterpret_cast<const float4*>(leafmom + (long)l * kMomStride);
        const float2 m1 = *reinterpret_cast<const float2*>(leafmom + (long)l * kMomStride + 4);
        const double Q = (double)m0.x + (double)m0.y;
        const double mx = m0.z, my = m0.w, mz = m1.x, mt = m1.y;
        const double cx = (compact3((uint32_t)l) + 0.5) * h - half_box, cy = (compact3((uint32_t)l >> 1) + 0.5) * h - half_box,
                     cz = (compact3((uint32_t)l >> 2) + 0.5) * h - half_box;
        a[0] += Q;
        a[1] += mx + Q * cx;
        a[2] += my + Q * cy;
        a[3] += mz + Q * cz;
        a[4] += mt + 2.0 * (cx * mx + cy * my + cz * mz) + Q * (cx * cx + cy * cy + cz * cz);
    }
    for (int c = 0; c < 5; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int c = 0; c < 5; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 5) partial[5 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// warp j computes root row j: M0_j = sum_c sum_k A_c[j][k] M1_c[k] in FP64
__global__ void k_root(int nc, int ncp, int depth, const double* __restrict__ Ad, const float* __restrict__ M1,
                       const float* __restrict__ M0, double* __restrict__ root) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (j >= nc) return;
    double s = 0.0;
    if (depth == 0) {
        s = (lane == 0) ? (double)M0[j] : 0.0;
    } else {
        for (int e = lane; e < 8 * nc; e += 32) {
            const int c = e / nc, k = e - c * nc;
            s += Ad[((long)c * nc + j) * nc + k] * (double)M1[(long)c * ncp + k];
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) root[j] = s;
}

// L0 = Lambda M0 (FP64), written as the FP32 level-0 local expansion.  Block 0 also totals
// Q, D, T from the fixed-order partials and leaves c2 (Q, D, T), c2 = 2 pi / (3 V), in FP32 for
// the per-atom correction (qdtf).
__global__ void k_lattice(int nc, int ncp, const double* __restrict__ Lam, double* __restrict__ root,
                          float* __restrict__ L0, double c2, float* __restrict__ qdtf) {
    if (blockIdx.x == 0 && threadIdx.x < 5) {
        const double* partial = root + nc + 8;
        double t = 0.0;
        for (int b = 0; b < kQdtBlocks; ++b) t += partial[5 * b + threadIdx.x];
        root[nc + threadIdx.x] = t;
        qdtf[threadIdx.x] = (float)(c2 * t);
    }
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (j >= ncp) return;
    double s = 0.0;
    if (j < nc)
        for (int k = lane; k < nc; k += 32) s += Lam[(long)j * nc + k] * root[k];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) L0[j] = (float)s;
}

// ---- M2L, FP32 CUDA cores: a tile of target boxes of one level and octant class ----
constexpr int kM2LTB = 16;
struct LevelOffsets {
    long off[kMaxDepth + 1];
};

__global__ void k_m2l_fp32(const M2LTile* __restrict__ tiles, int nc, int ncp, const float* __restrict__ TT,
                           const float* __restrict__ M, float* __restrict__ L, LevelOffsets lo,
                           int periodic) {
    extern __shared__ float ms[];  // [TB][ncp]
    const M2LTile t = tiles[blockIdx.x];
    const int lev = t.level, cls = t.cls, np = t.nparents;
    const int nb = 1 << lev;
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = (cls >> 2) & 1;
    const float* Ml = M + lo.off[lev] * ncp;
    float* Ll = L + lo.off[lev] * ncp;
    const int j = threadIdx.x;
    float acc[kM2LTB];
#pragma unroll
    for (int g = 0; g < kM2LTB; ++g) acc[g] = 0.f;
    for (int idx = 0; idx < 216; ++idx) {
        const int ox = idx / 36 - 2 - cx, oy = (idx / 6) % 6 - 2 - cy, oz = idx % 6 - 2 - cz;
        if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
        __syncthreads();
        for (int e = threadIdx.x; e < kM2LTB * ncp; e += blockDim.x) {
            const int g = e / ncp, k = e - g * ncp;
            float v = 0.f;
            if (g < np) {
                const uint32_t b = ((uint32_t)(t.parent0 + g) << 3) | (uint32_t)cls;
                int sx = (int)compact3(b) + ox, sy = (int)compact3(b >> 1) + oy, sz = (int)compact3(b >> 2) + oz;
                bool ok = true;
                if (periodic) {
                    sx &= nb - 1;
                    sy &= nb - 1;
                    sz &= nb - 1;
                } else {
                    ok = sx >= 0 && sx < nb && sy >= 0 && sy < nb && sz >= 0 && sz < nb;
                }
                if (ok) v = Ml[(long)morton3(sx, sy, sz) * ncp + k];
            }
            ms[e] = v;
        }
        __syncthreads();
        const float* top = TT + (long)((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)) * ncp * ncp + j;
        for (int k = 0; k < nc; ++k) {
            const float tv = top[(long)k * ncp];
#pragma unroll
            for (int g = 0; g < kM2LTB; ++g) acc[g] = fmaf(tv, ms[g * ncp + k], acc[g]);
        }
    }
    for (int g = 0; g < np; ++g) {
        const uint32_t b = ((uint32_t)(t.parent0 + g) << 3) | (uint32_t)cls;
        Ll[(long)b * ncp + j] = acc[g];
    }
}

// ---- M2L, FP32 CUDA cores, register-blocked: a brick of target boxes of one level and class ----
// The target boxes of octant class c form an n^3 sub-grid (n = 2^(level-1)); a source at offset
// o of a target lies in class pi = (c + o) mod 2 at sub-grid displacement delta = (c + o - pi) / 2
// in {-1, 0, 1}^3, so for fixed (c, pi) every delta maps the brick onto the brick shifted by
// delta in the pi sub-grid.  A CTA owns a brick of up to 4 x 4 x 8 = 128 target boxes and all
// output coefficients (ncp <= 128).  Per (source class pi, chunk of kF32KC input coefficients) it
// stages the brick's source halo ((bx + 2)(by + 2)(bz + 2) boxes, periodic images or zeros) in
// shared memory; per valid delta it stages the operator chunk T_o[k][j] and every thread adds
// T x M for its 8 output coefficients x 8 boxes (64 FP32 accumulators, 64 FMAs per k).  Target
// boxes outside the interaction list's near field only: no ghost-row work.  T is the bank
// [op][k][j] (j = output coefficient, fastest).  A CTA takes one (brick, source class pi) pair
// -- eight times as many CTAs as bricks, so that the waves on the SMs are nearly full -- and
// writes its partial local expansions to part[pi]; k_sum8 adds the eight partials in a fixed
// order into L.
constexpr int kF32KC = 16;
// The source halo of a 4 x 4 x 8 brick (6 x 6 x 10 boxes) in shared memory, three times: copy s
// holds the boxes z + s at z, so that a thread's pencil of 8 boxes at any z shift is two aligned
// 16-byte loads.  A pencil row is 12 floats (16-byte aligned), a plane 80 floats (the 8 pencils
// of a warp then fall in 8 distinct 4-bank groups).
constexpr int kF32Row = 12, kF32Plane = 80;
constexpr int kF32Halo = 6 * kF32Plane;
struct F32Smem {
    float hs[3][kF32KC][kF32Halo];
    __align__(16) float ts[2][kF32KC][128];
};

void f32_bricks(int lmin, int depth, std::vector<F32Brick>& out) {
    out.clear();
    for (int l = lmin; l <= depth; ++l) {
        const int n = 1 << (l - 1);
        // every brick is 4 x 4 x 8 boxes (those beyond n, on coarse levels, are computed and
        // dropped), so that a thread's 8 boxes are 8 consecutive halo entries
        const int bx = 4, by = 4, bz = 8;
        for (int c = 0; c < 8; ++c)
            for (int i0 = 0; i0 < n; i0 += bx)
                for (int j0 = 0; j0 < n; j0 += by)
                    for (int k0 = 0; k0 < n; k0 += bz) out.push_back({l, c, i0, j0, k0, bx, by, bz});
    }
}

// ---- packed two-wide FP32 arithmetic (f32x2) ----
__device__ __forceinline__ unsigned long long f2pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2unpack(unsigned long long v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__global__ void __launch_bounds__(256, 2) k_m2l_f32(const F32Brick* __restrict__ bricks, int ncp,
                                                    const float* __restrict__ T, const float* __restrict__ M,
                                                    float* __restrict__ part, long part_stride, LevelOffsets lo,
                                                    int periodic) {
    extern __shared__ __align__(16) unsigned char f32_smem[];
    F32Smem& sm = *reinterpret_cast<F32Smem*>(f32_smem);
    auto& ts = sm.ts;
    const F32Brick br = bricks[blockIdx.x];
    const int n = 1 << (br.level - 1);
    const int cx = br.cls & 1, cy = (br.cls >> 1) & 1, cz = (br.cls >> 2) & 1;
    constexpr int hy = 6, hz = 10, nh = 6 * 6 * 10;  // halo of a 4 x 4 x 8 brick
    const float* Ml = M + lo.off[br.level] * ncp;
    const int tid = threadIdx.x;
    // coefficients 8 tc .. +7, boxes 8 tb .. +7 of the brick.  A warp holds 4 coefficient groups x
    // 8 box groups: its operator loads (two 16-byte reads per k) then fall in one 128-byte
    // wavefront, and its 8 box pencils ((i * 6 + j) * 10 floats apart in the halo) in 8 distinct
    // banks, so shared-memory traffic per k stays below the FMA time.
    const int w = tid >> 5, lane = tid & 31;
    const int tc = 4 * (w & 3) + (lane & 3), tb = 8 * (w >> 2) + (lane >> 2);
    const bool cact = 8 * tc < ncp;
    // the thread's 8 boxes are the pencil (i, j) = (tb / 4, tb % 4), k = 0..7: halo row of plane
    // i + dx + 1, row j + dy + 1, entries dz + 1 .. dz + 8 (copy dz + 1 from its start)
    const int hb0 = (tb >> 2) * kF32Plane + (tb & 3) * kF32Row;
    // accumulators in coefficient pairs (2 a, 2 a + 1) x 8 boxes, updated with f32x2 FMAs: half
    // the FMA instructions of scalar code for the same FMA-pipe work; every element is still one
    // FP32 FMA per term, in the same order
    unsigned long long acc2[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc2[a][e] = 0ull;
    const int nkc = ncp / kF32KC;
    const int pi = blockIdx.y;
    {
        const int px = pi & 1, py = (pi >> 1) & 1, pz = (pi >> 2) & 1;
        for (int kc = 0; kc < nkc; ++kc) {
            __syncthreads();  // the previous chunk's readers are done with hs and ts
            // source halo of this (pi, kc): kF32KC consecutive coefficients per box
            for (int h = tid; h < nh * kF32KC; h += 256) {
                const int kk = h % kF32KC, hbx = h / kF32KC;
                const int hk = hbx % hz, hj = (hbx / hz) % hy, hi = hbx / (hz * hy);
                int si = br.i0 + hi - 1, sj = br.j0 + hj - 1, sk = br.k0 + hk - 1;
                bool ok = true;
                if (periodic) {
                    si = (si + n) & (n - 1);
                    sj = (sj + n) & (n - 1);
                    sk = (sk + n) & (n - 1);
                } else {
                    ok = si >= 0 && si < n && sj >= 0 && sj < n && sk >= 0 && sk < n;
                }
                float v = 0.f;
                if (ok) v = Ml[(long)morton3(2 * si + px, 2 * sj + py, 2 * sk + pz) * ncp + kc * kF32KC + kk];
                const int q = hi * kF32Plane + hj * kF32Row + hk;
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3)
                    if (hk >= c3) sm.hs[c3][kk][q - c3] = v;
            }
            // the valid shifts of (c, pi): a bit per delta; operator chunks double-buffered --
            // the next shift's chunk is read into registers while the current one is used
            unsigned vmask = 0;
            for (int d = 0; d < 27; ++d) {
                const int ox = 2 * (d / 9 - 1) + px - cx, oy = 2 * ((d / 3) % 3 - 1) + py - cy, oz = 2 * (d % 3 - 1) + pz - cz;
                if (abs(ox) > 1 || abs(oy) > 1 || abs(oz) > 1) vmask |= 1u << d;
            }
            const int nq = kF32KC * ncp / 4;  // float4 of one operator chunk
            auto chunk_src = [&](int d) {
                const int ox = 2 * (d / 9 - 1) + px - cx, oy = 2 * ((d / 3) % 3 - 1) + py - cy, oz = 2 * (d % 3 - 1) + pz - cz;
                return reinterpret_cast<const float4*>(
                    T + ((long)((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)) * ncp + kc * kF32KC) * ncp);
            };
            float4 pre[2];
            auto fetch = [&](int d) {
                const float4* src = chunk_src(d);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = tid + 256 * r;
                    pre[r] = q < nq ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            };
            auto stash = [&](int buf) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = tid + 256 * r;
                    if (q < nq) reinterpret_cast<float4*>(&ts[buf][q / (ncp / 4)][0])[q % (ncp / 4)] = pre[r];
                }
            };
            unsigned m = vmask;
            int d = __ffs(m) - 1;
            m &= m - 1;
            fetch(d);
            stash(0);
            __syncthreads();  // the halo and the first operator chunk are in place
            int cur = 0;
            while (d >= 0) {
                const int dn = m ? __ffs(m) - 1 : -1;
                m &= m - 1;
                if (dn >= 0) fetch(dn);
                const int dx = d / 9 - 1, dy = (d / 3) % 3 - 1, dz = d % 3 - 1;
                const int so = (dx + 1) * kF32Plane + (dy + 1) * kF32Row;
                const float* hcopy = &sm.hs[dz + 1][0][0];
                if (cact) {
#pragma unroll 8
                    for (int k = 0; k < kF32KC; ++k) {
                        const float4 a0 = *reinterpret_cast<const float4*>(&ts[cur][k][8 * tc]);
                        const float4 a1 = *reinterpret_cast<const float4*>(&ts[cur][k][8 * tc + 4]);
                        const unsigned long long A0 = f2pack(a0.x, a0.y), A1 = f2pack(a0.z, a0.w),
                                                 A2 = f2pack(a1.x, a1.y), A3 = f2pack(a1.z, a1.w);
                        const float4* hrow = reinterpret_cast<const float4*>(hcopy + k * kF32Halo + hb0 + so);
                        const float4 b0 = hrow[0], b1 = hrow[1];
                        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const unsigned long long B = f2pack(bv[e], bv[e]);
                            acc2[0][e] = f2fma(A0, B, acc2[0][e]);
                            acc2[1][e] = f2fma(A1, B, acc2[1][e]);
                            acc2[2][e] = f2fma(A2, B, acc2[2][e]);
                            acc2[3][e] = f2fma(A3, B, acc2[3][e]);
                        }
                    }
                }
                if (dn >= 0) stash(cur ^ 1);
                __syncthreads();  // the next chunk is in place; nobody reads this one any more
                cur ^= 1;
                d = dn;
            }
        }
    }
    if (!cact) return;
    float* Ll = part + (long)pi * part_stride + lo.off[br.level] * ncp;
    const int ti = br.i0 + (tb >> 2), tj = br.j0 + (tb & 3);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int tk = br.k0 + e;
        if (ti >= n || tj >= n || tk >= n) continue;  // padding of a coarse level's brick
        const uint32_t box = morton3(2 * ti + cx, 2 * tj + cy, 2 * tk + cz);
        float4* dst = reinterpret_cast<float4*>(Ll + (long)box * ncp + 8 * tc);
        const float2 c0 = f2unpack(acc2[0][e]), c1 = f2unpack(acc2[1][e]), c2 = f2unpack(acc2[2][e]),
                     c3 = f2unpack(acc2[3][e]);
        dst[0] = make_float4(c0.x, c0.y, c1.x, c1.y);
        dst[1] = make_float4(c2.x, c2.y, c3.x, c3.y);
    }
}

// L[i] = sum_{pi = 0..7} part[pi][i] in this order, over n floats (float4 vectors)
__global__ void k_sum8(long n4, const float4* __restrict__ part, long stride4, float4* __restrict__ L) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
        float4 s = part[i];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            const float4 v = part[q * stride4 + i];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        L[i] = s;
    }
}

// ---- L2P: potential and gradient of the leaf local expansion at u (units of h) ----
template <int P>
__device__ __forceinline__ void l2p_eval(const float* __restrict__ Lb, float x, float y, float z, float& phi,
                                         float& gx, float& gy, float& gz) {
    phi = gx = gy = gz = 0.f;
    regular_harmonics<P>(x, y, z, [&](int n, int m, float pr, float pi) {
        const float w = (m == 0) ? 1.f : 2.f;
        const float Lr = (m == 0) ? __ldg(Lb + n * n) : __ldg(Lb + n * n + 2 * m - 1);
        const float Li = (m == 0) ? 0.f : __ldg(Lb + n * n + 2 * m);
        phi += w * (Lr * pr - Li * pi);
        if (n < P) {
            const int q1 = (n + 1) * (n + 1);
            const float apr = __ldg(Lb + q1 + 2 * (m + 1) - 1), api = __ldg(Lb + q1 + 2 * (m + 1));
            float cr, ci, br, bi;
            if (m == 0) {
                cr = __ldg(Lb + q1);
                ci = 0.f;
                br = -apr;  // L_{n+1}^{-1} = -conj(L_{n+1}^{1})
                bi = api;
            } else {
                cr = __ldg(Lb + q1 + 2 * m - 1);
                ci = __ldg(Lb + q1 + 2 * m);
                if (m == 1) {
                    br = __ldg(Lb + q1);
                    bi = 0.f;
                } else {
                    br = __ldg(Lb + q1 + 2 * (m - 1) - 1);
                    bi = __ldg(Lb + q1 + 2 * (m - 1));
                }
            }
            const float c1 = c_g1[n][m], c2 = c_g2[n][m], c3 = c_g3[n][m];
            const float Ar = c1 * apr, Ai = c1 * api, Br = c2 * br, Bi = c2 * bi;
            const float hw = 0.5f * w;
            gx += hw * ((Ar - Br) * pr - (Ai - Bi) * pi);
            gy += hw * ((Ar + Br) * pi + (Ai + Bi) * pr);
            gz += w * c3 * (cr * pr - ci * pi);
        }
    });
}

struct NearParams {
    int n, nleaf, depth, periodic, use_far, ncp;
    float h, Lbox, ke;
    const uint32_t* start;
    const uint32_t* count;
    const float4* pos;
    const float* Lleaf;
    const float* qdtf;  // c2 (Q, Dx, Dy, Dz, T), c2 = 2 pi / (3 V) (periodic) or null
    const uint32_t* perm;
    float* F;
    float* phi_out;
    float* phis;
    float2* epart;  // per-block sum of q phi as a compensated (hi, lo) pair; totalled in FP64 by k_final
    int* status;     // device status word (FMM_DEV_TIMEOUT when a near-field staging wait expires)
    long long wlim;       // bound of the near field's staging waits (clock cycles)
    int leaves_per_warp;  // consecutive target leaves of each near-field warp
    const int2* items;    // work items (leaf, tile) of the leaves above kNearTile atoms, count in items[0].x
    int items_cap;
    int lose_copies;      // test hook (fmm_inject_copy_loss): staging copies announced, not issued
};

// Outputs per atom, one thread per atom in leaf order: the far field (L2P of the leaf's local
// expansion plus the periodic background term) added to the near field from k_p2p, then F in
// input order, phi, the sorted potential, and the block's partial sum of q phi: a fixed-order
// tree over the block's 128 atoms in compensated FP32 (exact products by FMA, TwoSum at every
// level), kept as a (hi, lo) pair that k_final totals in FP64.
constexpr int kOutThreads = 128;
__device__ __forceinline__ float2 two_sum(float a, float b) {  // a + b = s + e exactly
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}
template <int P>
__global__ void __launch_bounds__(kOutThreads) k_far_out(int n, int use_far, NearParams a,
                                                         const uint32_t* __restrict__ skey,
                                                         const float4* __restrict__ near) {
    __shared__ float2 red[kOutThreads];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float2 e = make_float2(0.f, 0.f);
    if (s < n) {
        const uint32_t leaf = skey[s];
        const bool leaf_ok = FMM_IN(leaf, a.nleaf);
        const float h = a.h;
        const float cx = (compact3(leaf) + 0.5f) * h, cy = (compact3(leaf >> 1) + 0.5f) * h,
                    cz = (compact3(leaf >> 2) + 0.5f) * h;
        const float4 me = a.pos[s];
        float pot = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        if (use_far && leaf_ok) {
            const float ih = 1.0f / h;
            l2p_eval<P>(a.Lleaf + (long)leaf * a.ncp, (me.x - cx) * ih, (me.y - cy) * ih, (me.z - cz) * ih, pot, gx,
                        gy, gz);
            pot *= ih;
            gx *= ih * ih;
            gy *= ih * ih;
            gz *= ih * ih;
        }
        if (a.periodic && a.qdtf) {
            const float cq = a.qdtf[0], cdx = a.qdtf[1], cdy = a.qdtf[2], cdz = a.qdtf[3], ctr = a.qdtf[4];
            const float hb = 0.5f * a.Lbox;
            const float ux = me.x - hb, uy = me.y - hb, uz = me.z - hb;
            pot += cq * (ux * ux + uy * uy + uz * uz) - 2.f * (ux * cdx + uy * cdy + uz * cdz) + ctr;
            gx += 2.f * (cq * ux - cdx);
            gy += 2.f * (cq * uy - cdy);
            gz += 2.f * (cq * uz - cdz);
        }
        const float4 nr = near[s];
        pot += nr.x;
        gx += nr.y;
        gy += nr.z;
        gz += nr.w;
        const int i = (int)a.perm[s];
        const float q = me.w;
        if (a.F && FMM_IN(i, n)) {
            a.F[3L * i] = -a.ke * q * gx;
            a.F[3L * i + 1] = -a.ke * q * gy;
            a.F[3L * i + 2] = -a.ke * q * gz;
        }
        if (a.phi_out && FMM_IN(i, n)) a.phi_out[i] = a.ke * pot;
        a.phis[s] = pot;
        const float qp = q * pot;
        e = make_float2(qp, fmaf(q, pot, -qp));
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int d = kOutThreads / 2; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) {
            const float2 u = red[threadIdx.x], v = red[threadIdx.x + d];
            const float2 t = two_sum(u.x, v.x);
            red[threadIdx.x] = make_float2(t.x, t.y + (u.y + v.y));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) a.epart[blockIdx.x] = red[0];
}

// ---- Hamiltonian interpolation: the intra-site correction ----
// With forms X of a site and their weights w_X (two forms: (1 - lambda, lambda); four forms:
// the bilinear weights of (lambda_p, lambda_t), Sec. 2.1 Eq. 1 and Eq. 2), q_i = sum_X w_X q^X_i.
// Interpolating the Hamiltonian instead of the charges changes the pair term of atoms i, j of
// one site by C_ij = sum_X w_X q^X_i q^X_j - q_i q_j = sum_X w_X (q^X_i - q_i)(q^X_j - q_j)
// (for two forms lambda (1 - lambda) dq_i dq_j), i = j with the self-image term psi_0, and
// dC_ij/dl = sum_X (dw_X/dl)(q^X_i - q_i)(q^X_j - q_j).  psi is the pair potential the FMM
// sums: 1/r open; periodic, psi(r) = 1/|r| + sum over the 26 neighbouring images 1/|r - nL|
// + c2 |r|^2 + h(r), with c2 = 2 pi / 3V and h the lattice remainder, evaluated as the root
// local expansion of a unit charge at the root centre (the lattice operator's first column)
// at u = r / L.
struct HiParams {
    int n, K, periodic, nforms;
    float L, ke, c2;
    const float* coef;  // h, normalised root local expansion (periodic)
    const int* site_ptr;
    const int* site_atoms;
    const uint32_t* inv;
    const float4* pos;
    const float* q[4];  // the forms, input order
    const float* lam;   // [K] or [2K]
    float* F;           // input order, corrected in place (may be null)
    double* site_out;   // [K][3]: energy, dV/dlambda(_p), dV/dlambda_t corrections
    float4* g_h;        // input order, per form X: sum_{j} (q^X_j - q_j) psi_ij (j = i: psi_0)
};

// psi(r) - [self ? 1/|r| : 0] and its gradient in r; r = 0 with self gives psi_0
template <int P>
__device__ void hi_pair(const HiParams& p, float rx, float ry, float rz, bool self, float& psi, float& gx,
                        float& gy, float& gz) {
    psi = gx = gy = gz = 0.f;
    if (!self) {
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float ri = 1.0f / sqrtf(r2);
        const float ri3 = ri * ri * ri;
        psi = ri;
        gx = -rx * ri3;
        gy = -ry * ri3;
        gz = -rz * ri3;
    }
    if (!p.periodic) return;
    const float L = p.L;
    for (int n = 0; n < 27; ++n) {
        if (n == 13) continue;
        const float dx = rx - (float)(n / 9 - 1) * L, dy = ry - (float)((n / 3) % 3 - 1) * L,
                    dz = rz - (float)(n % 3 - 1) * L;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float ri = 1.0f / sqrtf(r2);
        const float ri3 = ri * ri * ri;
        psi += ri;
        gx -= dx * ri3;
        gy -= dy * ri3;
        gz -= dz * ri3;
    }
    psi += p.c2 * (rx * rx + ry * ry + rz * rz);
    gx += 2.f * p.c2 * rx;
    gy += 2.f * p.c2 * ry;
    gz += 2.f * p.c2 * rz;
    const float iL = 1.0f / L;
    float hp, hx, hy, hz;
    l2p_eval<P>(p.coef, rx * iL, ry * iL, rz * iL, hp, hx, hy, hz);
    psi += hp * iL;
    gx += hx * iL * iL;
    gy += hy * iL * iL;
    gz += hz * iL * iL;
}

// the forms' deviations q^X - q of atom `ia` under weights w (unused forms: 0)
__device__ __forceinline__ void hi_dev(const HiParams& p, int ia, const float* w, float* dev) {
    float Q[4] = {0.f, 0.f, 0.f, 0.f}, q = 0.f;
    for (int X = 0; X < p.nforms; ++X) {
        Q[X] = p.q[X][ia];
        q = fmaf(w[X], Q[X], q);
    }
#pragma unroll
    for (int X = 0; X < 4; ++X) dev[X] = X < p.nforms ? Q[X] - q : 0.f;
}

// one warp per site, one lane per site atom: each lane sums over the other atoms of its site
// (every pair is evaluated from both sides, so no atomics and a fixed order)
template <int P>
__global__ void __launch_bounds__(128) k_hi(HiParams p) {
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (k >= p.K) return;
    const int a0 = p.site_ptr[k], na = p.site_ptr[k + 1] - a0;
    float w[4] = {0.f, 0.f, 0.f, 0.f}, wp[4] = {0.f, 0.f, 0.f, 0.f}, wt[4] = {0.f, 0.f, 0.f, 0.f};
    if (p.nforms == 4) {
        const float lp = p.lam[2 * k], lt = p.lam[2 * k + 1];
        w[0] = (1.f - lp) * (1.f - lt), w[1] = (1.f - lp) * lt, w[2] = lp * (1.f - lt), w[3] = lp * lt;
        wp[0] = -(1.f - lt), wp[1] = -lt, wp[2] = 1.f - lt, wp[3] = lt;
        wt[0] = -(1.f - lp), wt[1] = 1.f - lp, wt[2] = -lp, wt[3] = lp;
    } else {
        const float l = p.lam[k];
        w[0] = 1.f - l, w[1] = l;
        wp[0] = -1.f, wp[1] = 1.f;
    }
    float psi0, t0, t1, t2;
    hi_pair<P>(p, 0.f, 0.f, 0.f, true, psi0, t0, t1, t2);
    double e = 0.0, ep = 0.0, et = 0.0;
    for (int a = lane; a < na; a += 32) {
        const int ia = p.site_atoms[a0 + a];
        if (!FMM_IN(ia, p.n) || !FMM_IN(p.inv[ia], p.n)) continue;  // (no shuffle inside this loop)
        const float4 pa = p.pos[p.inv[ia]];
        float da[4];
        hi_dev(p, ia, w, da);
        float c = 0.f, cp = 0.f, ct = 0.f, g[4];
#pragma unroll
        for (int X = 0; X < 4; ++X) {
            c = fmaf(w[X], da[X] * da[X], c);
            cp = fmaf(wp[X], da[X] * da[X], cp);
            ct = fmaf(wt[X], da[X] * da[X], ct);
            g[X] = da[X] * psi0;
        }
        float sc = c * psi0, scp = cp * psi0, sct = ct * psi0;  // 2 x (this atom's energy share)
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int b = 0; b < na; ++b) {
            if (b == a) continue;
            const int ib = p.site_atoms[a0 + b];
            if (!FMM_IN(ib, p.n) || !FMM_IN(p.inv[ib], p.n)) continue;
            const float4 pb = p.pos[p.inv[ib]];
            float db[4];
            hi_dev(p, ib, w, db);
            float rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
            if (p.periodic) {  // minimum image: the truncated h is most accurate for small |r|
                rx -= p.L * rintf(rx / p.L);
                ry -= p.L * rintf(ry / p.L);
                rz -= p.L * rintf(rz / p.L);
            }
            float psi, hx, hy, hz;
            hi_pair<P>(p, rx, ry, rz, false, psi, hx, hy, hz);
            float cab = 0.f, cpab = 0.f, ctab = 0.f;
#pragma unroll
            for (int X = 0; X < 4; ++X) {
                const float pr = da[X] * db[X];
                cab = fmaf(w[X], pr, cab);
                cpab = fmaf(wp[X], pr, cpab);
                ctab = fmaf(wt[X], pr, ctab);
                g[X] = fmaf(db[X], psi, g[X]);
            }
            sc = fmaf(cab, psi, sc);
            scp = fmaf(cpab, psi, scp);
            sct = fmaf(ctab, psi, sct);
            gx = fmaf(cab, hx, gx);
            gy = fmaf(cab, hy, gy);
            gz = fmaf(cab, hz, gz);
        }
        if (p.F) {
            p.F[3L * ia] -= p.ke * gx;
            p.F[3L * ia + 1] -= p.ke * gy;
            p.F[3L * ia + 2] -= p.ke * gz;
        }
        p.g_h[ia] = make_float4(g[0], g[1], g[2], g[3]);
        e += 0.5 * (double)sc;
        ep += 0.5 * (double)scp;
        et += 0.5 * (double)sct;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, d);
        ep += __shfl_xor_sync(0xffffffffu, ep, d);
        et += __shfl_xor_sync(0xffffffffu, et, d);
    }
    if (lane == 0) {
        p.site_out[3 * k] = (double)p.ke * e;
        p.site_out[3 * k + 1] = (double)p.ke * ep;
        p.site_out[3 * k + 2] = (double)p.ke * et;
    }
}

template <int P>
static void launch_hi(const HiParams& hp, cudaStream_t st) {
    k_hi<P><<<(hp.K + 3) / 4, 128, 0, st>>>(hp);
}

// Near field (P2P).  Each warp takes a run of consecutive target leaves (one by default).
// (1) Staging: lanes 0..26 resolve the 27 neighbour leaves of a leaf (periodic image shift,
//     start, count) and keep them in registers; the target's own leaf is segment 0, its count
//     rounded up to even.  A warp scan gives each segment's offset in the warp's buffer, and lane
//     o copies segment o with one cp.async.bulk (a leaf's atoms are contiguous in leaf order),
//     completing on the buffer's mbarrier.  While a warp waits, the other resident warps (five
//     per SM sub-partition) keep the FMA pipe busy.
// (2) After the (bounded) wait: the image shift added to the wrapped segments, zero-charge pads
//     far away in the odd slots, then the atoms repacked in place into pairs
//     (x0 x1 y0 y1 | z0 z1 q0 q1) for the f32x2 arithmetic.
// (3) Work mapping: tp target pairs (two targets per lane) x np source pairs.  Each target pair
//     gets k source slices (source pairs j, j + k, j + 2k, ...); slice g = j tp + t runs on lane
//     g mod 32 in phase g / 32 (slice-major: the lanes of a quarter warp mostly read the same
//     source pair, a broadcast).  (phases, k) comes from a table that minimises phases x slice
//     length, and every lane of a phase runs the same trip count, so lanes never diverge in the
//     pair loop.  Only the own leaf's pairs need the r > 0 test (self, coincident atoms), since
//     equal positions always share a leaf.  After each phase a fixed shuffle tree adds each
//     target's slice sums and the owner lane of the target pair adds the result: a fixed order,
//     so results are bitwise reproducible for every block shape.
// A leaf whose neighbourhood does not fit the buffer (kNearCap atoms) stages it in rounds, and
// leaves above kNearTile atoms are split into work items of kNearTile targets listed by the
// binning (near_item, near_big).  k_far_out adds the far field and writes the outputs.
constexpr int kNearCap = 592;                   // staged atoms per buffer (neighbourhood + 2 pads)
constexpr int kNearMaxPairs = kNearCap / 2;     // source pairs of a staged neighbourhood
constexpr long long kNearWait = 4000000000LL;  // default bound of the staging wait (clock cycles, about 2 s)
__device__ __forceinline__ float rsqrt_approx(float x) {  // MUFU reciprocal square root
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct NearWarpSmem {
    float4 buf[kNearCap];  // the staging buffer: AoS (x, y, z, q) as copied, then packed pairs
    uint64_t bar;          // completion of its bulk copies
};

// Work mapping of a leaf: for tpg target pairs (1..32) and np source pairs (1..kNearMaxPairs),
// the phases P, slices per target pair k and slice length n = ceil(np / k) minimising
// P x (n + 3) (the 3 stands for a phase's own work: targets, slice sums), packed
// P | k << 3 | n << 11; and the multipliers rcp[d] = ceil(2^20 / d), d <= 128, so that
// a / d = (a rcp[d]) >> 20 exactly for the small dividends of the mapping (a < 2^20 / d).
struct NearMapTable {
    uint32_t map[32][kNearMaxPairs];
    uint32_t rcp[129];
};
constexpr NearMapTable near_map_table() {
    NearMapTable t{};
    for (int tpg = 1; tpg <= 32; ++tpg)
        for (int np = 1; np <= kNearMaxPairs; ++np) {
            int best = 1 << 30, P = 1, k = 1, n = np;
            for (int pc = 1; pc <= 4; ++pc) {
                int kc = (32 * pc) / tpg;
                kc = kc > np ? np : (kc < 1 ? 1 : kc);
                const int nc = (np + kc - 1) / kc;
                if (pc * (nc + 3) < best) {
                    best = pc * (nc + 3);
                    P = pc;
                    k = kc;
                    n = nc;
                }
            }
            t.map[tpg - 1][np - 1] = (uint32_t)(P | k << 3 | n << 11);
        }
    for (int d = 1; d <= 128; ++d) t.rcp[d] = (uint32_t)(((1u << 20) + d - 1) / d);
    return t;
}
__constant__ NearMapTable c_near = near_map_table();
__device__ __forceinline__ int near_div(int a, int d) {  // a / d for 0 <= a < 2^20 / d, d <= 128
    return (int)(((uint32_t)a * c_near.rcp[d]) >> 20);
}

__device__ __forceinline__ void near_output(float4* __restrict__ near, int s, float pot, float gx, float gy,
                                            float gz) {
    near[s] = make_float4(pot, gx, gy, gz);
}

// Sums of one source pair (A = (x0 x1 y0 y1), B = (z0 z1 q0 q1)) at two targets: the potential
// q/r and the gradient of q/r at the target, q (s - x) / r^3.
template <bool kCheck>
__device__ __forceinline__ void near_step(const float4 A, const float4 B, const unsigned long long (&mx)[2],
                                          const unsigned long long (&my)[2], const unsigned long long (&mz)[2],
                                          unsigned long long (&P)[2], unsigned long long (&X)[2],
                                          unsigned long long (&Y)[2], unsigned long long (&Z)[2]) {
    const unsigned long long sx = f2pack(A.x, A.y), sy = f2pack(A.z, A.w), sz = f2pack(B.x, B.y),
                             sq = f2pack(B.z, B.w);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const unsigned long long dx = f2sub(sx, mx[r]), dy = f2sub(sy, my[r]), dz = f2sub(sz, mz[r]);
        const float2 r2 = f2unpack(f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx))));
        float r0 = rsqrt_approx(r2.x), r1 = rsqrt_approx(r2.y);
        if (kCheck) {  // the self pair and coincident atoms
            r0 = (r2.x > 0.f) ? r0 : 0.f;
            r1 = (r2.y > 0.f) ? r1 : 0.f;
        }
        const unsigned long long ri = f2pack(r0, r1);
        const unsigned long long qri = f2mul(sq, ri);
        P[r] = f2add(P[r], qri);
        const unsigned long long qri3 = f2mul(qri, f2mul(ri, ri));
        X[r] = f2fma(qri3, dx, X[r]);
        Y[r] = f2fma(qri3, dy, Y[r]);
        Z[r] = f2fma(qri3, dz, Z[r]);
    }
}

// A leaf's staging, held in registers: lane o < 27 keeps segment o (first sorted atom, atom
// count, offset in the buffer, image shift); the counts and the mask are the same in every lane.
struct NearStage {
    int s0, sc, off;
    float shx, shy, shz;
    int cnt, total;  // own atoms, total slots (own leaf padded to even)
    unsigned wrap;   // segments with a nonzero image shift
};

// (1), the segment table of `leaf`: lane o < 27 gets neighbour segment o (segment 0 = the own
// leaf), its offset in a buffer that holds all of them (the own leaf padded to even).
__device__ __forceinline__ NearStage near_segments(const NearParams& a, int lane, int leaf) {
    const int nb = 1 << a.depth;
    NearStage t{0, 0, 0, 0.f, 0.f, 0.f, 0, 0, 0u};
    if (lane < 27) {  // lane 0 = own leaf (offset 13), lanes 1..26 = the others
        const int o = (lane == 0) ? 13 : (lane <= 13 ? lane - 1 : lane);
        const int sx = (int)compact3(leaf) + o / 9 - 1, sy = (int)compact3(leaf >> 1) + (o / 3) % 3 - 1,
                  sz = (int)compact3(leaf >> 2) + o % 3 - 1;
        const int wx = sx & (nb - 1), wy = sy & (nb - 1), wz = sz & (nb - 1);  // periodic wrap
        if (a.periodic || (sx == wx && sy == wy && sz == wz)) {
            const uint32_t src = morton3(wx, wy, wz);
            t.s0 = (int)a.start[src];
            t.sc = (int)a.count[src];
            if (!FMM_OK(t.s0 >= 0 && t.s0 + t.sc <= a.n)) t.sc = 0;  // an empty segment instead
            t.shx = (float)(sx - wx) * a.h;
            t.shy = (float)(sy - wy) * a.h;
            t.shz = (float)(sz - wz) * a.h;
        }
    }
    const int slot = (lane == 0) ? ((t.sc + 1) & ~1) : t.sc;  // own leaf padded to even
    int incl = slot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    t.off = incl - slot;
    t.total = __shfl_sync(0xffffffffu, incl, 31);
    t.cnt = __shfl_sync(0xffffffffu, t.sc, 0);
    t.wrap = __ballot_sync(0xffffffffu, lane < 27 && t.sc > 0 && (t.shx != 0.f || t.shy != 0.f || t.shz != 0.f));
    return t;
}

// (1): the segment table of `leaf` and, when the neighbourhood fits a buffer, the bulk copies of
// its segments into buf, completing on bar.  The caller has ordered the buffer's earlier
// generic-proxy accesses before these asynchronous writes.
__device__ __forceinline__ NearStage near_stage(const NearParams& a, float4* buf, uint64_t* bar, int lane,
                                                int leaf) {
    const NearStage t = near_segments(a, lane, leaf);
    // nothing to stage without targets, or for a leaf that k_p2p_big takes
    const bool staged = t.cnt > 0 && t.cnt <= kNearTile && ((t.total + 1) & ~1) <= kNearCap;
    if (lane == 0) tc::mbar_arrive_expect_tx(bar, staged ? 16u * (uint32_t)(t.total - (t.cnt & 1)) : 0u);
    __syncwarp();
    if (staged && lane < 27 && t.sc > 0 && !a.lose_copies && FMM_OK(t.off + t.sc <= kNearCap))
        tc::bulk_g2s(buf + t.off, a.pos + t.s0, 16u * (uint32_t)t.sc, bar);
    return t;
}

// (3) for a staged source list: the phases of target-pair slices over the source pairs
// [sb, sb + np) of buf, of which the first nck may be own pairs (the r > 0 test); the targets
// are the own leaf's pairs at the start of buf.  Writes the outputs of the leaf's cnt target
// atoms (sorted slots st ..), or adds to them (add: a later round of the same leaf).
__device__ __forceinline__ void near_phases(const float4* buf, int lane, int cnt, int st, int sb, int np, int nck,
                                            bool add, float4* __restrict__ near) {
    const int tp = (cnt + 1) >> 1;
    for (int tg = 0; tg < tp; tg += 32) {  // groups of up to 32 target pairs
        const int tpg = min(32, tp - tg);
        const uint32_t m = c_near.map[tpg - 1][np - 1];
        const int P = (int)(m & 7u), k = (int)((m >> 3) & 255u), n = (int)(m >> 11);
        const int nslices = tpg * k;
        const int nchk = min(n - 1, near_div(nck + k - 1, k));  // steps whose pairs may be own
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        for (int ph = 0; ph < P; ++ph) {
            const int g = ph * 32 + lane;
            const bool act = g < nslices;
            const int jg = near_div(g, tpg);
            const int t = act ? g - jg * tpg : 0, j = act ? jg : 0;
            const bool full = act && j + (n - 1) * k < np;  // this slice has n source pairs
            const float4 TA = buf[2 * (tg + t)], TB = buf[2 * (tg + t) + 1];
            unsigned long long mx[2], my[2], mz[2], Pv[2], Xv[2], Yv[2], Zv[2];
            mx[0] = f2pack(TA.x, TA.x);
            mx[1] = f2pack(TA.y, TA.y);
            my[0] = f2pack(TA.z, TA.z);
            my[1] = f2pack(TA.w, TA.w);
            mz[0] = f2pack(TB.x, TB.x);
            mz[1] = f2pack(TB.y, TB.y);
#pragma unroll
            for (int r = 0; r < 2; ++r) Pv[r] = Xv[r] = Yv[r] = Zv[r] = 0ull;
            const float4* sp = buf + 2 * (sb + j);
            const int stride = 2 * k;
            int i = 0;
            for (; i < nchk; ++i, sp += stride) near_step<true>(sp[0], sp[1], mx, my, mz, Pv, Xv, Yv, Zv);
            if (i < n - 1) {  // steps i .. n - 2 exist for every lane: sources loaded a step ahead
                float4 pa = sp[0], pb = sp[1];
#pragma unroll 2
                for (; i + 1 < n - 1; ++i) {
                    sp += stride;
                    const float4 na = sp[0], nb = sp[1];
                    near_step<false>(pa, pb, mx, my, mz, Pv, Xv, Yv, Zv);
                    pa = na;
                    pb = nb;
                }
                near_step<false>(pa, pb, mx, my, mz, Pv, Xv, Yv, Zv);
                ++i;
                sp += stride;
            }
            if (full) {  // the last source pair of the slices that have n
                if ((n - 1) * k < nck) near_step<true>(sp[0], sp[1], mx, my, mz, Pv, Xv, Yv, Zv);
                else near_step<false>(sp[0], sp[1], mx, my, mz, Pv, Xv, Yv, Zv);
            }
            // slice sums of this phase: lane l holds slice (t, j) with l = j tpg + t - 32 ph, so a
            // target's slices sit tpg lanes apart from lane l mod tpg on; a fixed tree over them
            // leaves the phase sum on that first lane, and the owner lane of the target adds it
            float v[8];
            {
                const float2 p0 = f2unpack(Pv[0]), x0 = f2unpack(Xv[0]), y0 = f2unpack(Yv[0]), z0 = f2unpack(Zv[0]);
                const float2 p1 = f2unpack(Pv[1]), x1 = f2unpack(Xv[1]), y1 = f2unpack(Yv[1]), z1 = f2unpack(Zv[1]);
                v[0] = p0.x + p0.y, v[1] = x0.x + x0.y, v[2] = y0.x + y0.y, v[3] = z0.x + z0.y;
                v[4] = p1.x + p1.y, v[5] = x1.x + x1.y, v[6] = y1.x + y1.y, v[7] = z1.x + z1.y;
            }
            const int m = near_div(lane, tpg);  // this lane's place among its target's lanes
            for (int d = 1; d * tpg < 32; d <<= 1) {
                const bool take = (m & (2 * d - 1)) == 0 && lane + d * tpg < 32 && g + d * tpg < nslices;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float o = __shfl_down_sync(0xffffffffu, v[e], d * tpg);
                    if (take) v[e] += o;
                }
            }
            {
                const int ph0 = ph * 32 - near_div(ph * 32, tpg) * tpg;  // (32 ph) mod tpg
                const int src = lane >= ph0 ? lane - ph0 : lane - ph0 + tpg;  // first lane of target `lane`
                const bool has = lane < tpg && ph * 32 + src < nslices;
                float u[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) u[e] = __shfl_sync(0xffffffffu, v[e], src & 31);
                if (has) {
                    acc0.x += u[0];
                    acc0.y += u[1];
                    acc0.z += u[2];
                    acc0.w += u[3];
                    acc1.x += u[4];
                    acc1.y += u[5];
                    acc1.z += u[6];
                    acc1.w += u[7];
                }
            }
        }
        if (lane < tpg) {
            const int t0 = 2 * (tg + lane);
            if (add) {  // a later round of the same leaf: add to the earlier rounds' sums
                const float4 u = near[st + t0];
                acc0 = make_float4(u.x + acc0.x, u.y + acc0.y, u.z + acc0.z, u.w + acc0.w);
                if (t0 + 1 < cnt) {
                    const float4 v = near[st + t0 + 1];
                    acc1 = make_float4(v.x + acc1.x, v.y + acc1.y, v.z + acc1.z, v.w + acc1.w);
                }
            }
            near_output(near, st + t0, acc0.x, acc0.y, acc0.z, acc0.w);
            if (t0 + 1 < cnt) near_output(near, st + t0 + 1, acc1.x, acc1.y, acc1.z, acc1.w);
        }
    }
}


// (2) and (3) for one staged leaf in buf: image shifts of the wrapped segments, pads, packed
// pairs, then the phases of target-pair slices; writes the leaf's near-field outputs.
__device__ __forceinline__ void near_leaf(const NearParams& a, const NearStage& T, float4* buf, int lane,
                                          float4* __restrict__ near) {
    const int cnt = T.cnt, total = T.total;
    const int npairs = (total + 1) >> 1;
    for (unsigned wm = T.wrap; wm; wm &= wm - 1) {
        const int o = __ffs(wm) - 1;
        const int o0 = __shfl_sync(0xffffffffu, T.off, o), no = __shfl_sync(0xffffffffu, T.sc, o);
        const float ax = __shfl_sync(0xffffffffu, T.shx, o), ay = __shfl_sync(0xffffffffu, T.shy, o),
                    az = __shfl_sync(0xffffffffu, T.shz, o);
        for (int j = lane; j < no; j += 32) {
            float4 v = buf[o0 + j];
            v.x += ax;
            v.y += ay;
            v.z += az;
            buf[o0 + j] = v;
        }
    }
    // a zero charge far away contributes nothing (own leaf odd, list odd)
    if (lane == 0 && (cnt & 1)) buf[cnt] = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
    if (lane == 1 && (total & 1)) buf[total] = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);
    __syncwarp();
    for (int j = lane; j < npairs; j += 32) {
        const float4 A = buf[2 * j], B = buf[2 * j + 1];
        buf[2 * j] = make_float4(A.x, B.x, A.y, B.y);
        buf[2 * j + 1] = make_float4(A.z, B.z, A.w, B.w);
    }
    __syncwarp();
    near_phases(buf, lane, cnt, __shfl_sync(0xffffffffu, T.s0, 0), 0, npairs, __shfl_sync(0xffffffffu, T.off, 1) >> 1,
                false, near);
}

// One work item of the near field: the targets t0 .. t0 + kNearTile - 1 of `leaf` (at most
// kNearTile) at the start of the buffer, and the neighbourhood -- the own leaf first, then the
// other 26 segments, as one list -- staged in rounds of the remaining room, a segment split
// across rounds where it does not fit.  Every round runs the phases of the staged near field over
// its source pairs (the own leaf's pairs with the r > 0 test); later rounds add to the outputs
// the earlier ones wrote, in round order.  It serves the leaves above kNearTile atoms (one item
// per tile, listed by the binning) and the smaller leaves whose neighbourhood does not fit the
// buffer in one piece (one item).  buf and bar: the warp's staging buffer and its initialised
// mbarrier, ph the count of its completed phases; returns false when a wait expired
// (FMM_DEV_TIMEOUT is set and nothing is left copying).
__device__ __noinline__ bool near_item(const NearParams& a, float4* buf, uint64_t* bar, uint32_t& ph, int lane,
                                       int leaf, int t0, float4* __restrict__ near) {
    const float4 pad = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f);  // a zero charge far away
    const NearStage T = near_segments(a, lane, leaf);
    const int cnt = T.cnt;
    const int tcnt = min(kNearTile, cnt - t0);
    if (tcnt <= 0) return true;  // (a stale item: cannot happen after a binning of this call)
    const int tslot = (tcnt + 1) & ~1, tpairs = tslot >> 1;
    const int room = kNearCap - tslot - 2;  // source atoms of one round (its pad included)
    const int st = __shfl_sync(0xffffffffu, T.s0, 0) + t0;
    const int own = cnt;  // the own leaf is the first stretch of the source list
    // the sources as one list: segment o at [excl, excl + sc)
    const int mine = lane < 27 ? T.sc : 0;
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int excl = incl - mine, total = __shfl_sync(0xffffffffu, incl, 31);
    for (int r0 = 0, r = 0; r0 < total; r0 += room, ++r) {
        const int r1 = min(r0 + room, total), ra = r1 - r0;
        // this lane's piece of its segment in the round
        const int lo = max(excl, r0), hi = min(excl + mine, r1);
        const bool has = lane < 27 && hi > lo;
        tc::fence_proxy_async();  // the warp's earlier reads and writes of the buffer first
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_expect_tx(bar, 16u * (uint32_t)(ra + (r == 0 ? tcnt : 0)));
        __syncwarp();
        if (r == 0 && lane == 0) tc::bulk_g2s(buf, a.pos + st, 16u * (uint32_t)tcnt, bar);
        if (has && FMM_OK(tslot + (hi - r0) <= kNearCap))  // (a skipped copy ends in the bounded wait)
            tc::bulk_g2s(buf + tslot + (lo - r0), a.pos + T.s0 + (lo - excl), 16u * (uint32_t)(hi - lo), bar);
        if (!tc::mbar_wait_all(bar, ph & 1u, a.wlim)) {
            if (lane == 0) atomicOr(a.status, FMM_DEV_TIMEOUT);
            tc::mbar_wait_all(bar, ph & 1u, kNearWait);  // nothing may still be copying when the warp exits
            return false;
        }
        ++ph;
        // image shifts of the wrapped pieces, pads, packed pairs
        const unsigned wm0 = T.wrap & __ballot_sync(0xffffffffu, has);
        for (unsigned wm = wm0; wm; wm &= wm - 1) {
            const int o = __ffs(wm) - 1;
            const int plo = __shfl_sync(0xffffffffu, lo, o), phi = __shfl_sync(0xffffffffu, hi, o);
            const float ax = __shfl_sync(0xffffffffu, T.shx, o), ay = __shfl_sync(0xffffffffu, T.shy, o),
                        az = __shfl_sync(0xffffffffu, T.shz, o);
            for (int j = plo + lane; j < phi; j += 32) {
                float4 v = buf[tslot + (j - r0)];
                v.x += ax;
                v.y += ay;
                v.z += az;
                buf[tslot + (j - r0)] = v;
            }
        }
        if (r == 0 && lane == 0 && (tcnt & 1)) buf[tcnt] = pad;
        if (lane == 1 && (ra & 1)) buf[tslot + ra] = pad;
        __syncwarp();
        const int np_r = (ra + 1) >> 1;
        for (int j = (r == 0 ? 0 : tpairs) + lane; j < tpairs + np_r; j += 32) {
            const float4 A = buf[2 * j], B = buf[2 * j + 1];
            buf[2 * j] = make_float4(A.x, B.x, A.y, B.y);
            buf[2 * j + 1] = make_float4(A.z, B.z, A.w, B.w);
        }
        __syncwarp();
        // source pairs of this round that may hold own atoms: those before the own leaf's end
        const int own_r = max(0, min(own, r1) - r0);
        near_phases(buf, lane, tcnt, st, tpairs, np_r, (own_r + 1) >> 1, r > 0, near);
        __syncwarp();
    }
    return true;
}

// The items of the leaves above kNearTile atoms (listed by the binning): warps first, first +
// stride, ... take them in turn (the grid does not know their number).
__device__ __forceinline__ void near_big(const NearParams& a, float4* buf, uint64_t* bar, uint32_t ph, int lane,
                                         int first, int stride, float4* __restrict__ near) {
    const int2* __restrict__ items = a.items;
    if (!items || first >= a.items_cap) return;  // no list (a handle without atoms) or nothing for this warp
    const int nitems = min(items[0].x, a.items_cap);
    for (int item = first; item < nitems; item += stride) {
        const int2 it = items[1 + item];
        if (!FMM_IN(it.x, a.nleaf)) continue;  // (the warp's lanes read the same item)
        if (!near_item(a, buf, bar, ph, lane, it.x, it.y * kNearTile, near)) return;
    }
}

// W warps per block: 1, 2 or 4 (the near-field block shape the autotuner picks; a block keeps
// its shared memory until its last warp is done).  Each warp takes leaves_per_warp consecutive
// leaves, waits for each leaf's copies while the other resident warps keep the FMA pipe busy,
// then takes its turn at the big leaves' items; the blocks after the leaves' (when the leaves'
// warps are fewer than kNearBigWarps) take only items.
template <int W>
__global__ void __launch_bounds__(32 * W, 20 / W) k_p2p(NearParams a, float4* __restrict__ near) {
    extern __shared__ __align__(128) unsigned char near_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    NearWarpSmem& S = reinterpret_cast<NearWarpSmem*>(near_smem)[w];
    const int leaf_blocks = (a.nleaf + W * a.leaves_per_warp - 1) / (W * a.leaves_per_warp);
    const int gw = blockIdx.x * W + w, gstride = gridDim.x * W;
    if (lane == 0) {
        tc::mbar_init(&S.bar, 1);
        tc::fence_mbar_init();
    }
    __syncwarp();
    uint32_t ph = 0;  // completed phases of the warp's mbarrier
    if ((int)blockIdx.x < leaf_blocks) {
        const int first = gw * a.leaves_per_warp;
        const int last = min(a.nleaf, first + a.leaves_per_warp);
        for (int leaf = first; leaf < last; ++leaf) {
            if (leaf > first) {  // this leaf's copies overwrite what the warp read and wrote before
                tc::fence_proxy_async();
                __syncwarp();
            }
            const NearStage cur = near_stage(a, S.buf, &S.bar, lane, leaf);
            if (!tc::mbar_wait_all(&S.bar, ph & 1u, a.wlim)) {
                if (lane == 0) atomicOr(a.status, FMM_DEV_TIMEOUT);
                // nothing may still be copying when the warp exits (with lost copies nothing is)
                if (!a.lose_copies) tc::mbar_wait_all(&S.bar, ph & 1u, kNearWait);
                return;
            }
            ++ph;
            if (cur.cnt > 0 && cur.cnt <= kNearTile) {  // larger leaves: their items
                if (2 * ((cur.total + 1) >> 1) <= kNearCap) {
                    near_leaf(a, cur, S.buf, lane, near);
                } else if (!near_item(a, S.buf, &S.bar, ph, lane, leaf, 0, near)) {  // in rounds
                    return;
                }
            }
            __syncwarp();
        }
    }
    near_big(a, S.buf, &S.bar, ph, lane, gw, gstride, near);
}

// Grid of the near field: W warps per block, leaves_per_warp consecutive leaves per warp, and at
// least kNearBigWarps warps in all for the items of the big leaves (the extra ones return at once
// when there are none).  Measured at 500,000 atoms: one leaf per warp and one warp per block
// (0.135 ms alone) beat two staging buffers per warp at 2, 4 or 8 leaves per warp (0.160-0.186
// ms: eleven warps per SM left the pair loop latency-bound) and four warps per block (0.143 ms).
constexpr int kNearLeavesPerWarp = 1;
constexpr int kNearBigWarps = 148 * 8;
template <int W>
static void launch_p2p(NearParams a, float4* near, cudaStream_t st) {
    a.leaves_per_warp = kNearLeavesPerWarp;
    const int per_block = W * kNearLeavesPerWarp;
    const int leaf_blocks = (a.nleaf + per_block - 1) / per_block;
    const int item_warps = std::min(a.items_cap, kNearBigWarps) - leaf_blocks * W;
    const int big_blocks = item_warps > 0 ? (item_warps + W - 1) / W : 0;
    k_p2p<W><<<leaf_blocks + big_blocks, 32 * W, (size_t)W * sizeof(NearWarpSmem), st>>>(a, near);
}

// Per handle, with its device current: the dynamic shared-memory limits of the near field
// (every block shape) and of the FP32 M2L.
void near_configure(Handle* h) {
    (void)h;
    cudaFuncSetAttribute(k_m2l_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(F32Smem));
    constexpr int smem = (int)sizeof(NearWarpSmem);
    cudaFuncSetAttribute(k_p2p<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_p2p<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * smem);
    cudaFuncSetAttribute(k_p2p<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * smem);
}

// E = 1/2 k sum of the per-block partials of q phi, totalled in FP64: each of the
// kFinalBlocks blocks sums a fixed slice, and the last block to finish (atomic ticket) adds the
// block totals in block order, so the result is deterministic.  dV/dlambda_k = k sum over the
// site's atoms of dq phi (FP64), one warp per site in a fixed order.
constexpr int kFinalBlocks = 32;
static_assert(8 + 5 * kQdtBlocks + 4 + kFinalBlocks + 1 <= kRootDoubles, "root scratch layout");
__global__ void __launch_bounds__(256) k_final(int n, int nparts, const float2* __restrict__ epart, double ke,
                                               double* __restrict__ E, int K, int ncoord,
                                               const int* __restrict__ site_ptr,
                                               const int* __restrict__ site_atoms, const uint32_t* __restrict__ inv,
                                               const float* __restrict__ dq, const float* __restrict__ dqt,
                                               const float* __restrict__ phis, float* __restrict__ dVdl,
                                               double* __restrict__ blocksum, unsigned int* __restrict__ ticket,
                                               const double* __restrict__ hi_site) {
    __shared__ double red[256];
    __shared__ bool last;
    const int per = (nparts + kFinalBlocks - 1) / kFinalBlocks;
    const int b0 = blockIdx.x * per, b1 = min(nparts, b0 + per);
    double s = 0.0;
    for (int i = b0 + threadIdx.x; i < b1; i += 256) s += (double)epart[i].x + (double)epart[i].y;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        blocksum[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == kFinalBlocks - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int b = 0; b < kFinalBlocks; ++b) t += ((volatile double*)blocksum)[b];
        double hsum = 0.0;  // Hamiltonian interpolation: per-site corrections, in site order
        if (hi_site)
            for (int k = 0; k < K; ++k) hsum += hi_site[3 * k];
        if (E) E[0] = 0.5 * ke * t + hsum;
        *ticket = 0u;  // ready for the next call
    }
    // one warp per site: lane j sums the site's atoms j, j + 32, ... in order, then a fixed-order
    // shuffle tree adds the lanes (the site's atoms are loaded in parallel, not one after another)
    const int lane = threadIdx.x & 31;
    if (dVdl)
        for (int k = (blockIdx.x * 256 + threadIdx.x) >> 5; k < K; k += kFinalBlocks * 8) {
            double v = 0.0, vt = 0.0;  // dE/dlambda(_p), dE/dlambda_t
            for (int a = site_ptr[k] + lane; a < site_ptr[k + 1]; a += 32) {
                if (!FMM_IN(site_atoms[a], n) || !FMM_IN(inv[site_atoms[a]], n)) continue;  // (no shuffle in the loop)
                const uint32_t si = inv[site_atoms[a]];
                v += (double)dq[si] * (double)phis[si];
                if (ncoord == 2) vt += (double)dqt[si] * (double)phis[si];
            }
            for (int off = 16; off > 0; off >>= 1) {
                v += __shfl_down_sync(0xffffffffu, v, off);
                vt += __shfl_down_sync(0xffffffffu, vt, off);
            }
            if (lane == 0) {
                dVdl[ncoord * k] = (float)(ke * v + (hi_site ? hi_site[3 * k + 1] : 0.0));
                if (ncoord == 2) dVdl[2 * k + 1] = (float)(ke * vt + (hi_site ? hi_site[3 * k + 2] : 0.0));
            }
        }
}

struct ChargeGrads {
    float* q[4];  // dL/dq^X per form (any may be null)
};

// Reverse mode: gbar = dL/dE.  dE/dx = -F; dE/dlambda = dV/dlambda; dE/dq^X_i = k phi_i w_X
// for a site atom (w_X the weight of form X in q_i), plus k w_X g_h[i][X] with Hamiltonian
// interpolation; atoms outside every site have q_i = qA_i.
__global__ void k_adjoint(int n, int K, int ncoord, int nforms, const double* __restrict__ gbar,
                          const float* __restrict__ F, const float* __restrict__ phi, const float* __restrict__ dVdl,
                          const int32_t* __restrict__ site, const float* __restrict__ lam, float* __restrict__ gx,
                          ChargeGrads gq, float* __restrict__ glam, float ke, const float4* __restrict__ g_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float g = (float)gbar[0];
    if (i < ncoord * K && glam) glam[i] = dVdl[i] * g;
    if (i >= n) return;
    if (gx) {
        gx[3L * i] = -F[3L * i] * g;
        gx[3L * i + 1] = -F[3L * i + 1] * g;
        gx[3L * i + 2] = -F[3L * i + 2] * g;
    }
    const int s = site[i];
    float w[4] = {1.f, 0.f, 0.f, 0.f};
    if (s >= 0 && s < K) {
        if (nforms == 4) {
            const float lp = lam[2 * s], lt = lam[2 * s + 1];
            w[0] = (1.f - lp) * (1.f - lt), w[1] = (1.f - lp) * lt, w[2] = lp * (1.f - lt), w[3] = lp * lt;
        } else {
            w[0] = 1.f - lam[s], w[1] = lam[s];
        }
    }
    float hg[4] = {0.f, 0.f, 0.f, 0.f};
    if (g_h && s >= 0 && s < K) {
        const float4 t = g_h[i];
        hg[0] = t.x, hg[1] = t.y, hg[2] = t.z, hg[3] = t.w;
    }
    for (int X = 0; X < nforms; ++X)
        if (gq.q[X]) gq.q[X][i] = w[X] * (phi[i] + ke * hg[X]) * g;
}

// ---------------------------------------------------------------------------------------------
template <int P>
static void launch_p2m(int nleaf, float h, const Handle* hd, float* Mleaf, float* mom,
                       cudaStream_t st) {
    k_p2m<P><<<(nleaf + kP2mLeaves - 1) / kP2mLeaves, 128, 0, st>>>(nleaf, h, hd->start, hd->count, hd->pos,
                                                                     Mleaf, hd->ncp, mom, hd->n);
}
template <int P>
static void launch_far_out(int n, int use_far, const NearParams& a, const uint32_t* skey, const float4* near,
                           cudaStream_t st) {
    k_far_out<P><<<(n + kOutThreads - 1) / kOutThreads, kOutThreads, 0, st>>>(n, use_far, a, skey, near);
}

#define FMM_DISPATCH_P(p, FN, ...)         \
    switch (p) {                            \
        case 1: FN<1>(__VA_ARGS__); break;  \
        case 2: FN<2>(__VA_ARGS__); break;  \
        case 3: FN<3>(__VA_ARGS__); break;  \
        case 4: FN<4>(__VA_ARGS__); break;  \
        case 5: FN<5>(__VA_ARGS__); break;  \
        case 6: FN<6>(__VA_ARGS__); break;  \
        case 7: FN<7>(__VA_ARGS__); break;  \
        case 8: FN<8>(__VA_ARGS__); break;  \
        case 9: FN<9>(__VA_ARGS__); break;  \
        case 10: FN<10>(__VA_ARGS__); break; \
        case 11: FN<11>(__VA_ARGS__); break; \
        case 12: FN<12>(__VA_ARGS__); break; \
        case 13: FN<13>(__VA_ARGS__); break; \
        case 14: FN<14>(__VA_ARGS__); break; \
        default: break;                     \
    }


static inline int sort_passes(int depth) { return (3 * depth + 7) / 8; }


// K slices for a split-K translation whose output is tree level l: the work buffer holds
// 8^d ncp floats, so at most 8^(d-l) slices of that level's output fit; at most `want`.
static inline int split_slices(int d, int l, int want) {
    long cap = 1;
    for (int i = l; i < d && cap < want; ++i) cap *= 8;
    return (int)std::min<long>(cap, want);
}

// profiling: record the next pool event on `st` and return its index (-1 when not profiling)
static inline int mark(Handle* h, cudaStream_t st) {
    if (!h->profiling || h->ev_used >= kNumEvents) return -1;
    cudaEventRecord(h->ev[h->ev_used], st);
    return h->ev_used++;
}
static inline void span(Handle* h, int k, int a, int b) {
    h->stage_ev[k][0] = a;
    h->stage_ev[k][1] = b;
}

// L2L into tree level l from level l - 1, added to the M2L result already there
static void l2l_level(Handle* h, int l, cudaStream_t st) {
    const int np = 1 << (3 * (l - 1));
    if (h->l2l_tc.dev)  // coarse levels split over K (one chunk per block), summed in a fixed order
        translate_tc(h->l2l_tc, h->L + h->lvl_off[l - 1] * h->ncp, h->ncp, np, h->L + h->lvl_off[l] * h->ncp,
                     8 * h->ncp, true, h->status, st, split_slices(h->depth, l, 8), h->work, h->wait_limit,
                     (h->copy_loss & FMM_LOSE_TRANSLATE) != 0);
    else
        sgemm(np, 8 * h->ncp, h->ncp, h->L + h->lvl_off[l - 1] * h->ncp, h->ncp, h->B2, 8 * h->ncp,
              h->L + h->lvl_off[l] * h->ncp, 8 * h->ncp, true, st);
}

// The coarse levels (lmin .. depth - 2) get their own branch when the M2L runs on the tensor
// cores: their M2L, the periodic root and their L2L run on `side` concurrently with the M2L of
// the two finest levels, which dominates; only the L2L into the two finest levels follows it.
static inline int coarse_top(const Handle* h) {
    const int lmin = h->periodic ? 1 : 2;
    const bool tc = h->precision != FMM_FP32 && m2l_tc_supported(h) && h->ntiles > 0;
    return (tc && h->depth - 2 >= lmin) ? h->depth - 2 : -1;
}

int launches_per_eval(const Handle* h) {
    const int d = h->depth;
    int n = 4 /*count, scan, place, order+gather*/ + 1 /*p2m*/;
    const int lmin = h->periodic ? 1 : 2;
    if (d >= lmin) n += 2 * (d - lmin);  // M2M parent levels d-1 .. lmin (split-K product + sum)
    if (h->periodic) n += 3;       // Q/D/T partials + root + lattice
    if (d >= lmin)  // M2L: the coarse and the finest levels in two launches when split
        n += (h->precision != FMM_FP32 && m2l_tc_supported(h)) ? (coarse_top(h) >= 0 ? 2 : 1) * m2l_tc_launches(h)
             : (h->nbricks > 0 ? 2 : 1);  // FP32: the brick kernel and the sum of its partials
    if (d >= lmin) {  // L2L: coarse levels split over K (product + sum), the finest level in place
        const int lfirst = h->periodic ? 1 : lmin + 1;
        for (int l = lfirst; l <= d; ++l) n += (h->l2l_tc.dev && split_slices(d, l, 8) > 1) ? 2 : 1;
    }
    n += 1 /*p2p*/ + 1 /*far field + outputs*/ + 1 /*final*/;
    if (h->hamiltonian && h->K > 0) n += 1;  // intra-site correction
    return n;
}

// FP32 copies of c2 (Q, D, T) for the per-atom correction, after the FP64 totals and partials
static inline float* qdt_float(Handle* h) { return reinterpret_cast<float*>(h->root + h->nc + 8 + 5 * kQdtBlocks); }

int launch_eval(Handle* h, const float* x, double* E, float* F, float* dVdl, float* phi, cudaStream_t st) {
    const int n = h->n, d = h->depth, nb = 1 << d;
    const int nleaf = 1 << (3 * d);
    const float hleaf = (float)(h->box.edge / nb);
    BoxGeom g{h->box.origin[0], h->box.origin[1], h->box.origin[2], h->box.edge, h->s_bin, nb, d, h->periodic};
    const float* lam = h->lam_bound ? h->lam_bound : h->lam;
    h->ev_used = 0;
    for (auto& se : h->stage_ev) se[0] = se[1] = -1;
    TraceRange trace_eval("fmm:eval");
    const int e0 = mark(h, st);
    // --- binning: counting sort by leaf (see k_bin_count .. k_bin_order_gather) ---
    nvtxRangePushA("fmm:binning");
    const int ntiles = scan_tiles(nleaf);
    uint32_t* tilecnt = h->leafcnt + nleaf;  // [ntiles] atoms per tile of kScanTile leaves
    if (n > 0)
        k_bin_count<<<(n + kCountThreads - 1) / kCountThreads, kCountThreads, 0, st>>>(
            n, x, g, h->key, h->vA, h->leafcnt, ntiles, tilecnt, h->status, h->near_items);
    k_bin_scan<<<ntiles, kScanThreads, 0, st>>>(nleaf, h->leafcnt, tilecnt, h->start, h->count);
    h->perm = h->kA;
    h->sorted_key = h->kB;
    if (n > 0) {
        k_bin_place<<<(n + 255) / 256, 256, 0, st>>>(n, h->key, h->vA, h->start, h->vB, ntiles, tilecnt);
        ChargeForms cf{{h->qA, h->qB, h->qC, h->qD}, h->nforms, h->site, h->K, lam, h->dq, h->dqt};
        k_bin_order_gather<<<((nleaf + 1) / 2 + 3) / 4, 128, 0, st>>>(nleaf, h->start, h->count, h->vB, h->perm,
                                                            h->sorted_key, x, g, cf, h->pos, h->inv, h->status,
                                                            h->near_items, h->near_items_cap, n);
    }
    nvtxRangePop();
    // --- near field on the caller's stream, concurrent with the multipole chain ---
    NearParams a{};
    a.n = n;
    a.nleaf = nleaf;
    a.depth = d;
    a.periodic = h->periodic;
    a.use_far = h->periodic ? 1 : (d >= 2 ? 1 : 0);
    a.ncp = h->ncp;
    a.h = hleaf;
    a.Lbox = (float)h->box.edge;
    a.ke = (float)h->ke;
    a.start = h->start;
    a.count = h->count;
    a.pos = h->pos;
    a.Lleaf = h->L + h->lvl_off[d] * h->ncp;
    a.qdtf = h->periodic ? qdt_float(h) : nullptr;
    a.perm = h->perm;
    a.F = F;
    a.phi_out = phi;
    a.phis = h->phis;
    a.epart = h->epart;
    a.status = h->status;
    a.wlim = h->wait_limit > 0 ? h->wait_limit : kNearWait;
    a.items = h->near_items;
    a.items_cap = h->near_items_cap;
    a.lose_copies = (h->copy_loss & FMM_LOSE_NEAR) != 0;
    const int e1 = mark(h, st);
    span(h, 0, e0, e1);
    // fork: the chain P2M .. L2L on h->chain (highest priority), P2P here.  Serialised
    // profiling runs every stage on the eval's stream, one after the other, so that each
    // stage's events time its kernels alone.
    const bool serial = h->profiling == 2;
    cudaStream_t cs = serial ? st : h->chain;
    const int lc = coarse_top(h);  // top coarse level of the side branch, -1 without one
    cudaEventRecord(h->fork_ev, st);
    cudaStreamWaitEvent(cs, h->fork_ev, 0);
    nvtxRangePushA("fmm:near");
    if (h->p2p_warps == 1) launch_p2p<1>(a, h->near, st);
    else if (h->p2p_warps == 2) launch_p2p<2>(a, h->near, st);
    else launch_p2p<4>(a, h->near, st);
    nvtxRangePop();
    const int e1n = mark(h, st);
    span(h, 8, e1, e1n);
    const int e1c = serial ? e1n : e1;  // start of the chain's first stage
    // --- P2M ---
    float* Mleaf = h->M + h->lvl_off[d] * h->ncp;
    float* Lleaf = h->L + h->lvl_off[d] * h->ncp;
    nvtxRangePushA("fmm:P2M");
    FMM_DISPATCH_P(h->p, launch_p2m, nleaf, hleaf, h, Mleaf, h->periodic ? h->leafmom : nullptr, cs);
    nvtxRangePop();
    const int e2 = mark(h, cs);
    span(h, 1, e1c, e2);
    // --- M2M (FP32) for parent levels d-1 .. lmin: one GEMM per level,
    //     [parents x 8 ncp] (the 8 children are contiguous) x [8 ncp x ncp] ---
    const int lmin = h->periodic ? 1 : 2;
    nvtxRangePushA("fmm:M2M");
    for (int l = d - 1; l >= lmin; --l) {
        const int np = 1 << (3 * l);
        if (h->m2m_tc.dev)  // split K by child octant; coarse levels into up to 32 slices (their latency)
            translate_tc(h->m2m_tc, h->M + h->lvl_off[l + 1] * h->ncp, 8 * h->ncp, np, h->M + h->lvl_off[l] * h->ncp,
                         h->ncp, false, h->status, cs, split_slices(d, l, 32), h->work, h->wait_limit,
                         (h->copy_loss & FMM_LOSE_TRANSLATE) != 0);
        else
            sgemm(np, h->ncp, 8 * h->ncp, h->M + h->lvl_off[l + 1] * h->ncp, 8 * h->ncp, h->A, h->ncp,
                  h->M + h->lvl_off[l] * h->ncp, h->ncp, false, cs, 8, h->work);  // split K by child octant
    }
    nvtxRangePop();
    const int e3 = mark(h, cs);
    span(h, 2, e2, e3);
    // --- periodic root (FP64): root multipole, lattice operator, Q/D/T for the background term ---
    auto root = [&](cudaStream_t rs) {
        if (!h->periodic) return;
        TraceRange trace("fmm:root");
        const int nrowblk = (h->nc + 3) / 4;
        const float* M1 = (d >= 1) ? h->M + h->lvl_off[1] * h->ncp : nullptr;
        k_qdt<<<kQdtBlocks, 256, 0, rs>>>(nleaf, h->box.edge / nb, 0.5 * h->box.edge, h->leafmom, h->root + h->nc + 8);
        k_root<<<nrowblk, 128, 0, rs>>>(h->nc, h->ncp, d, h->Ad, M1, h->M, h->root);
        k_lattice<<<(h->ncp + 3) / 4, 128, 0, rs>>>(h->nc, h->ncp, h->Lam, h->root, h->L,
                                                     2.0 * M_PI / (3.0 * h->box.edge * h->box.edge * h->box.edge),
                                                     qdt_float(h));
    };
    // L2L: levels lmin+1 .. d (periodic: 1 .. d from the lattice-filled root)
    const int lfirst = h->periodic ? 1 : lmin + 1;
    if (lc >= 0) {
        // Side branch: the coarse levels' pack and M2L, the root, the coarse levels' L2L.  Their
        // M2L writes only levels lmin .. lc of L, the root only level 0, and the split-K work
        // buffer of their L2L is free: the M2M has finished and the chain's L2L waits for this.
        // The coarse M2L is issued first, so that its few CTAs run in the first wave and the
        // root and L2L after them fit beside the finest levels' tiles.  Neither M2L launch
        // waits for the near field: their CTAs take the SMs the near field's blocks leave, and
        // its remaining blocks run on the SMs the M2L's second wave leaves idle.
        cudaStream_t ss = serial ? st : h->side;
        cudaEventRecord(h->m2m_ev, cs);
        cudaStreamWaitEvent(ss, h->m2m_ev, 0);
        nvtxRangePushA("fmm:M2L coarse");
        launch_m2l_tc(h, ss, lmin, lc, kM2lPack);
        launch_m2l_tc(h, cs, lc + 1, d, kM2lPack);
        const int s0 = mark(h, ss);
        launch_m2l_tc(h, ss, lmin, lc, kM2lMma);
        nvtxRangePop();
        const int s1 = mark(h, ss);
        span(h, 9, s0, s1);
        root(ss);
        const int s2 = mark(h, ss);
        if (h->periodic) span(h, 3, s1, s2);
        nvtxRangePushA("fmm:L2L coarse");
        for (int l = lfirst; l <= lc; ++l) l2l_level(h, l, ss);
        nvtxRangePop();
        span(h, 10, s2, mark(h, ss));
        cudaEventRecord(h->side_ev, ss);
        // chain: the finest levels' M2L, then the L2L into them from the side branch's levels
        const int e4 = mark(h, cs);
        nvtxRangePushA("fmm:M2L");
        launch_m2l_tc(h, cs, lc + 1, d, kM2lMma);
        nvtxRangePop();
        const int e5 = mark(h, cs);
        span(h, 4, e4, e5);
        cudaStreamWaitEvent(cs, h->side_ev, 0);
        nvtxRangePushA("fmm:L2L");
        for (int l = std::max(lfirst, lc + 1); l <= d; ++l) l2l_level(h, l, cs);
        nvtxRangePop();
        span(h, 5, e5, mark(h, cs));
    } else {
        root(cs);
        const int e4 = mark(h, cs);
        if (h->periodic) span(h, 3, e3, e4);
        nvtxRangePushA("fmm:M2L");
        if (d >= lmin && h->ntiles > 0) {
            if (h->precision != FMM_FP32 && m2l_tc_supported(h)) {
                launch_m2l_tc(h, cs, lmin, d);
            } else {
                LevelOffsets lo{};
                for (int l = 0; l <= d; ++l) lo.off[l] = h->lvl_off[l];
                if (h->nbricks > 0) {
                    // partials of every level lmin .. d (the part of the level arrays from lmin on)
                    const long a0 = h->lvl_off[lmin] * h->ncp, n = (h->lvl_off[d + 1] - h->lvl_off[lmin]) * h->ncp;
                    const long stride = h->nbox_total * h->ncp;
                    k_m2l_f32<<<dim3(h->nbricks, 8), 256, sizeof(F32Smem), cs>>>(h->bricks, h->ncp, h->T, h->M,
                                                                                h->m2l_part, stride, lo, h->periodic);
                    k_sum8<<<std::min<long>((n / 4 + 255) / 256, 148L * 16), 256, 0, cs>>>(
                        n / 4, reinterpret_cast<const float4*>(h->m2l_part + a0), stride / 4,
                        reinterpret_cast<float4*>(h->L + a0));
                } else
                    k_m2l_fp32<<<h->ntiles, h->ncp, sizeof(float) * kM2LTB * h->ncp, cs>>>(
                        h->tiles, h->nc, h->ncp, h->T, h->M, h->L, lo, h->periodic);
            }
        }
        nvtxRangePop();
        const int e5 = mark(h, cs);
        span(h, 4, e4, e5);
        nvtxRangePushA("fmm:L2L");
        for (int l = lfirst; l <= d; ++l) l2l_level(h, l, cs);
        nvtxRangePop();
        span(h, 5, e5, mark(h, cs));
    }
    const int e6 = h->stage_ev[5][1];
    // join, then the far field and the outputs per atom
    cudaEventRecord(h->join_ev, cs);
    cudaStreamWaitEvent(st, h->join_ev, 0);
    nvtxRangePushA("fmm:far+outputs");
    if (n > 0) FMM_DISPATCH_P(h->p, launch_far_out, n, a.use_far, a, h->sorted_key, h->near, st);
    const bool hi = h->hamiltonian && h->K > 0;
    if (hi) {
        HiParams hp{};
        hp.n = n;
        hp.K = h->K;
        hp.periodic = h->periodic;
        hp.nforms = h->nforms;
        hp.q[0] = h->qA;
        hp.q[1] = h->qB;
        hp.q[2] = h->qC;
        hp.q[3] = h->qD;
        hp.L = (float)h->box.edge;
        hp.ke = (float)h->ke;
        hp.c2 = (float)(2.0 * M_PI / (3.0 * h->box.edge * h->box.edge * h->box.edge));
        hp.coef = h->hi_coef;
        hp.site_ptr = h->site_ptr;
        hp.site_atoms = h->site_atoms;
        hp.inv = h->inv;
        hp.pos = h->pos;
        hp.lam = lam;
        hp.F = F;
        hp.site_out = h->hi_site;
        hp.g_h = h->hi_g;
        FMM_DISPATCH_P(h->p, launch_hi, hp, st);
    }
    nvtxRangePop();
    const int e7 = mark(h, st);
    span(h, 6, e6, e7);
    const int nparts = (n + kOutThreads - 1) / kOutThreads;  // one q phi partial per output block
    double* fin = h->root + h->nc + 8 + 5 * kQdtBlocks + 4;  // [kFinalBlocks] block totals, then the ticket
    k_final<<<kFinalBlocks, 256, 0, st>>>(n, nparts, h->epart, h->ke, E, h->K, h->ncoord, h->site_ptr, h->site_atoms,
                                          h->inv, h->dq, h->dqt, h->phis, dVdl, fin,
                                          reinterpret_cast<unsigned int*>(fin + kFinalBlocks), hi ? h->hi_site : nullptr);
    span(h, 7, e7, mark(h, st));
    return 0;
}

// ---------------------------------------------------------------------------------------------
// Binning with no device allocation (fmm_binning_noalloc).
// The sort's scratch -- two key buffers, one value buffer and the digit table -- lives in a
// file-scope device array sized for FMM_NOALLOC_MAX_ATOMS atoms; every GPU that loads the
// library holds it until the process exits.  Calls share it, so calls that overlap on the GPU
// (different streams, no ordering between them) race; calls on one stream are ordered.
constexpr int kNoAllocSortBlocks = (FMM_NOALLOC_MAX_ATOMS + kSortTile - 1) / kSortTile;
constexpr size_t kNoAllocWords = 3ull * FMM_NOALLOC_MAX_ATOMS + 256ull * kNoAllocSortBlocks;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Device address of the scratch array on the current device.  Host code may not use the
// array's name as a device pointer (it is a host-side stand-in), so the address is looked up
// once per device, with that device current, and cached.
static fmm_status noalloc_scratch(uint32_t** out) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static uint32_t* addr[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FMM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FMM_ERR_CUDA;
        }
        addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = addr[dev];
    return FMM_OK;
}

extern "C" fmm_status fmm_binning_noalloc(const fmm_box* box, int periodic, int depth, int n, const float* x,
                                          uint32_t* key, uint32_t* perm, uint32_t* start, uint32_t* count,
                                          int* status, void* stream) {
    if (!box || !(box->edge > 0.0) || !std::isfinite(box->edge)) return FMM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(box->origin[a])) return FMM_ERR_ARG;
    if ((periodic != 0 && periodic != 1) || depth < 0 || depth > kMaxDepth) return FMM_ERR_ARG;
    if (n < 0 || n > FMM_NOALLOC_MAX_ATOMS) return FMM_ERR_ARG;  // beyond the static scratch
    if (!start || !count || (n > 0 && (!x || !key || !perm))) return FMM_ERR_ARG;
    uint32_t* scr = nullptr;
    fmm_status e = noalloc_scratch(&scr);
    if (e != FMM_OK) return e;
    uint32_t* kB = scr;
    uint32_t* kC = scr + FMM_NOALLOC_MAX_ATOMS;
    uint32_t* vS = scr + 2L * FMM_NOALLOC_MAX_ATOMS;
    uint32_t* table = scr + 3L * FMM_NOALLOC_MAX_ATOMS;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = 1 << depth, nleaf = 1 << (3 * depth);
    BoxGeom g{box->origin[0], box->origin[1], box->origin[2], box->edge, std::ldexp(1.0, depth) / box->edge,
              nb, depth, periodic};
    const int passes = sort_passes(depth);
    // values ping-pong between the scratch and the caller's perm so that the last pass lands in perm
    uint32_t* vbuf[2] = {(passes & 1) ? vS : perm, (passes & 1) ? perm : vS};
    cudaGetLastError();
    const uint32_t* kin = key;
    const uint32_t* vin = vbuf[0];
    if (n > 0) {
        k_keys<<<(n + 255) / 256, 256, 0, st>>>(n, x, g, key, vbuf[0], status);
        const int nblk = (n + kSortTile - 1) / kSortTile;
        uint32_t* kout[2] = {kB, kC};
        for (int ps = 0; ps < passes; ++ps) {
            uint32_t* ko = kout[ps & 1];
            uint32_t* vo = vbuf[(ps + 1) & 1];
            k_sort_hist<<<nblk, kSortThreads, 0, st>>>(n, kin, 8 * ps, table, nblk);
            k_sort_scan<<<1, 1024, 0, st>>>(table, 256 * nblk);
            k_sort_scatter<<<nblk, kSortThreads, 0, st>>>(n, kin, vin, ko, vo, 8 * ps, table, nblk);
            kin = ko;
            vin = vo;
        }
    }
    k_ranges<<<(nleaf + 255) / 256, 256, 0, st>>>(n, nleaf, kin, start, count);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

void launch_adjoint(Handle* h, const double* gbar, const float* F, const float* phi, const float* dVdl,
                    float* gx, float* const* gq, float* glam, cudaStream_t st) {
    const int m = h->n > h->ncoord * h->K ? h->n : h->ncoord * h->K;
    if (m == 0) return;
    const float* lam = h->lam_bound ? h->lam_bound : h->lam;
    ChargeGrads g{{gq[0], gq[1], h->nforms == 4 ? gq[2] : nullptr, h->nforms == 4 ? gq[3] : nullptr}};
    k_adjoint<<<(m + 255) / 256, 256, 0, st>>>(h->n, h->K, h->ncoord, h->nforms, gbar, F, phi, dVdl, h->site, lam, gx,
                                               g, glam, (float)h->ke, h->hamiltonian ? h->hi_g : nullptr);
}

}  // namespace fmmcph
