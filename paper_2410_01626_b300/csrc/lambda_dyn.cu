// Lambda dynamics on the device: one BAOAB Langevin step per titration site, driven by the
// force -dV/dlambda that fmm_eval returns, so a simulation loop needs no host round trip.
//
// The lambda particle has mass m and obeys m lambda'' = -dV/dlambda (Sec. 2.1, Eq. 1:
// F_lambda = -dH/dlambda; Sec. 2.7: m = 60 u, 2 fs steps).  Units: lambda dimensionless,
// time ps, energy kJ/mol, m in u (so m lambda'^2 is in kJ/mol).  Thermostat: Langevin with
// friction gamma (1/ps) at kT (kJ/mol), in the BAOAB splitting of Leimkuhler and Matthews.
// Reflecting walls keep lambda in [lo, hi].
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11), keyed by the seed,
// counter = (step, site); Gaussian pairs by the Box-Muller transform.  Counter based, so a
// trajectory is reproducible from (seed, step) alone and can resume from a checkpoint.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fmm_internal.h"

namespace fmmcph {

namespace {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    // round constants and Weyl increments of the published Philox4x32 definition
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += W0;
        k1 += W1;
    }
    return c;
}

__device__ __forceinline__ float uniform01(uint32_t u) {  // (0, 1]
    return ((float)(u >> 8) + 1.0f) * (1.0f / 16777216.0f);
}

__global__ void k_lambda_baoab(int K, float* __restrict__ lam, float* __restrict__ vel,
                               const float* __restrict__ dVdl, float dt, float inv_mass, float c1, float c2,
                               uint32_t seed_lo, uint32_t seed_hi, unsigned long long step, int first, float lo,
                               float hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float l = lam[k], v = vel[k];
    const float f = -dVdl[k];
    v += (first ? 0.5f : 1.0f) * dt * f * inv_mass;  // B (closing half of the last step + opening half)
    l += 0.5f * dt * v;                               // A
    const U4 r = philox4x32_10(U4{(uint32_t)step, (uint32_t)(step >> 32), (uint32_t)k, 0u}, seed_lo, seed_hi);
    const float u1 = uniform01(r.x), u2 = uniform01(r.y);
    const float xi = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    v = c1 * v + c2 * xi;                             // O
    l += 0.5f * dt * v;                               // A
    if (l < lo) {
        l = 2.f * lo - l;
        v = -v;
    }
    if (l > hi) {
        l = 2.f * hi - l;
        v = -v;
    }
    lam[k] = l;
    vel[k] = v;
}

}  // namespace

}  // namespace fmmcph

extern "C" fmm_status fmm_lambda_step(int n_sites, float* lambda, float* velocity, const float* dVdlambda, double dt,
                                      double mass, double gamma, double kT, unsigned long long seed,
                                      unsigned long long step, int first, double lo, double hi, void* stream) {
    if (n_sites < 0 || (n_sites > 0 && (!lambda || !velocity || !dVdlambda))) return FMM_ERR_ARG;
    if (!(dt > 0.0) || !(mass > 0.0) || !(gamma >= 0.0) || !(kT >= 0.0) || !(lo < hi)) return FMM_ERR_ARG;
    if (n_sites == 0) return FMM_OK;
    const double c1 = std::exp(-gamma * dt);
    const double c2 = std::sqrt((1.0 - c1 * c1) * kT / mass);
    cudaGetLastError();
    fmmcph::k_lambda_baoab<<<(n_sites + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        n_sites, lambda, velocity, dVdlambda, (float)dt, (float)(1.0 / mass), (float)c1, (float)c2,
        (uint32_t)seed, (uint32_t)(seed >> 32), step, first ? 1 : 0, (float)lo, (float)hi);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}
