// Tiled FP32 GEMM on CUDA cores for the dense translation steps (M2M, L2L):
//   C[M x N] (=|+=) A[M x K] B[K x N], all row-major, K and the leading dimensions
//   multiples of 4 (16-byte rows), N and M arbitrary.
// Tiles of BM x 128 outputs, BK = 16, 256 threads each computing TM x 4 outputs from
// shared-memory tiles (A stored k-major for broadcast reads), with the next K tile
// prefetched into registers while the current one is consumed.
#pragma once
#include <cuda_runtime.h>

namespace fmmcph {

// blockIdx.z selects one of gridDim.z equal slices of K; slice z writes (or adds) its partial
// product to C + z * cstride (split-K, summed afterwards in a fixed order by k_sum_slices).
template <int BM, int TM>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                               int accumulate, long cstride) {
    constexpr int BN = 128, BK = 16, TN = 4;
    {
        const int kslice = K / gridDim.z;
        A += (long)blockIdx.z * kslice;
        B += (long)blockIdx.z * kslice * ldb;
        C += (long)blockIdx.z * cstride;
        K = kslice;
    }
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    constexpr int A_F4 = BM * BK / 4;          // float4 elements of an A tile
    constexpr int A_LD = (A_F4 + 255) / 256;   // float4 loads of A per thread
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    float4 ra[A_LD], rb[2];
    auto load_tiles = [&](int k0) {
#pragma unroll
        for (int q = 0; q < A_LD; ++q) {
            const int e = tid + q * 256;          // BM rows x 4 float4
            const int r = e / (BK / 4), c4 = e % (BK / 4);
            const int gm = m0 + r, gk = k0 + c4 * 4;
            ra[q] = (e < A_F4 && gm < M && gk < K) ? *reinterpret_cast<const float4*>(A + (long)gm * lda + gk)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * 256;          // 16 rows x 32 float4
            const int r = e / (BN / 4), c4 = e % (BN / 4);
            const int gk = k0 + r, gn = n0 + c4 * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gk < K) {
                const float* bp = B + (long)gk * ldb + gn;
                if (gn + 3 < N) v = *reinterpret_cast<const float4*>(bp);
                else {
                    if (gn < N) v.x = bp[0];
                    if (gn + 1 < N) v.y = bp[1];
                    if (gn + 2 < N) v.z = bp[2];
                }
            }
            rb[q] = v;
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int q = 0; q < A_LD; ++q) {
            const int e = tid + q * 256;
            if (e >= A_F4) continue;
            const int r = e / (BK / 4), c4 = e % (BK / 4);
            As[buf][c4 * 4 + 0][r] = ra[q].x;
            As[buf][c4 * 4 + 1][r] = ra[q].y;
            As[buf][c4 * 4 + 2][r] = ra[q].z;
            As[buf][c4 * 4 + 3][r] = ra[q].w;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * 256;
            const int r = e / (BN / 4), c4 = e % (BN / 4);
            *reinterpret_cast<float4*>(&Bs[buf][r][c4 * 4]) = rb[q];
        }
    };

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    const int nk = (K + BK - 1) / BK;
    load_tiles(0);
    store_tiles(0);
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int buf = t & 1;
        if (t + 1 < nk) load_tiles((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; i += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + i]);
                a[i] = v.x;
                a[i + 1] = v.y;
                a[i + 2] = v.z;
                a[i + 3] = v.w;
            }
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN]);
            b[0] = bv.x;
            b[1] = bv.y;
            b[2] = bv.z;
            b[3] = bv.w;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < nk) store_tiles(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty * TM + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx * TN + j;
            if (gn >= N) continue;
            float* cp = C + (long)gm * ldc + gn;
            *cp = accumulate ? *cp + acc[i][j] : acc[i][j];
        }
    }
}

// C (=|+=) sum_z P_z, P_z = slice z of a split-K product, fixed summation order
__global__ void k_sum_slices(int M, int N, int ldc, int nz, const float* __restrict__ P, long pstride,
                             float* __restrict__ C, int accumulate) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)M * N) return;
    const int m = (int)(e / N), nn = (int)(e % N);
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += P[z * pstride + (long)m * N + nn];
    float* cp = C + (long)m * ldc + nn;
    *cp = accumulate ? *cp + s : s;
}

// C = A B (+C): chooses the row tile so that small-M problems still spread over the SMs.
// With `work` (>= ksplit * M * N floats) and ksplit > 1 the K range is split over blockIdx.z
// -- long, thin products are latency bound otherwise -- and summed in a fixed order.
inline void sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  bool accumulate, cudaStream_t st, int ksplit = 1, float* work = nullptr) {
    if (M <= 0 || N <= 0) return;
    const int nbn = (N + 127) / 128;
    const bool split = ksplit > 1 && work && K % (4 * ksplit) == 0;
    const int nz = split ? ksplit : 1;
    float* out = split ? work : C;
    const int ldo = split ? N : ldc;
    const long cst = split ? (long)M * N : 0;
    const int acc = split ? 0 : (accumulate ? 1 : 0);
    if ((long)((M + 63) / 64) * nbn * nz >= 148) {
        dim3 grid(nbn, (M + 63) / 64, nz);
        k_sgemm<64, 8><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, acc, cst);
    } else {
        dim3 grid(nbn, (M + 31) / 32, nz);
        k_sgemm<32, 4><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, acc, cst);
    }
    if (split) {
        const long tot = (long)M * N;
        k_sum_slices<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, ldc, nz, work, cst, C, accumulate ? 1 : 0);
    }
}

}  // namespace fmmcph
