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

#include <algorithm>
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

// dV_dw/dlambda of the double well (Sec. 2.2): b = [a0, a1, barrier, delta, kwall]
__device__ __forceinline__ float dw_slope(float l, const float* __restrict__ b) {
    const float a0 = b[0], a1 = b[1], h = b[2], d = b[3], kw = b[4];
    if (l < a0) return kw * (l - a0);
    if (l > a1) return kw * (l - a1);
    const float m = 0.5f * (a0 + a1);
    float va, vb, la, lb;
    if (l <= m) {
        va = 0.f, vb = h, la = a0, lb = m;
    } else {
        va = h, vb = d, la = m, lb = a1;
    }
    const float s = (l - la) / (lb - la);
    return (vb - va) * 6.f * s * (1.f - s) / (lb - la);
}

__global__ void k_lambda_baoab(int K, float* __restrict__ lam, float* __restrict__ vel,
                               const float* __restrict__ dVdl, const float* __restrict__ bias, float dt,
                               float inv_mass, float c1, float c2, uint32_t seed_lo, uint32_t seed_hi,
                               unsigned long long step, int first, float lo, float hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float l = lam[k], v = vel[k];
    float f = -dVdl[k];
    if (bias) f -= dw_slope(l, bias + 5L * k);
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

static fmm_status lambda_step(int n_sites, float* lambda, float* velocity, const float* dVdlambda,
                              const float* bias, double dt, double mass, double gamma, double kT,
                              unsigned long long seed, unsigned long long step, int first, double lo, double hi,
                              void* stream) {
    if (n_sites < 0 || (n_sites > 0 && (!lambda || !velocity || !dVdlambda))) return FMM_ERR_ARG;
    if (!(dt > 0.0) || !(mass > 0.0) || !(gamma >= 0.0) || !(kT >= 0.0) || !(lo < hi)) return FMM_ERR_ARG;
    if (n_sites == 0) return FMM_OK;
    const double c1 = std::exp(-gamma * dt);
    const double c2 = std::sqrt((1.0 - c1 * c1) * kT / mass);
    cudaGetLastError();
    fmmcph::k_lambda_baoab<<<(n_sites + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        n_sites, lambda, velocity, dVdlambda, bias, (float)dt, (float)(1.0 / mass), (float)c1, (float)c2,
        (uint32_t)seed, (uint32_t)(seed >> 32), step, first ? 1 : 0, (float)lo, (float)hi);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

extern "C" fmm_status fmm_lambda_step(int n_sites, float* lambda, float* velocity, const float* dVdlambda, double dt,
                                      double mass, double gamma, double kT, unsigned long long seed,
                                      unsigned long long step, int first, double lo, double hi, void* stream) {
    return lambda_step(n_sites, lambda, velocity, dVdlambda, nullptr, dt, mass, gamma, kT, seed, step, first, lo, hi,
                       stream);
}

extern "C" fmm_status fmm_lambda_step_bias(int n, float* lambda, float* velocity, const float* dVdlambda,
                                           const float* bias, double dt, double mass, double gamma, double kT,
                                           unsigned long long seed, unsigned long long step, int first, double lo,
                                           double hi, void* stream) {
    return lambda_step(n, lambda, velocity, dVdlambda, bias, dt, mass, gamma, kT, seed, step, first, lo, hi,
                       stream);
}

// ---- partition function correction (host, FP64) ----
namespace {

double dw_value(double l, double a0, double a1, double h, double d, double kw) {
    if (l < a0) return 0.5 * kw * (l - a0) * (l - a0);
    if (l > a1) return d + 0.5 * kw * (l - a1) * (l - a1);
    const double m = 0.5 * (a0 + a1);
    double va, vb, la, lb;
    if (l <= m) {
        va = 0.0, vb = h, la = a0, lb = m;
    } else {
        va = h, vb = d, la = m, lb = a1;
    }
    const double s = (l - la) / (lb - la);
    return va + (vb - va) * s * s * (3.0 - 2.0 * s);
}

// 64-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre recurrence)
struct GaussLegendre {
    double x[64], w[64];
    GaussLegendre() {
        const int n = 64;
        for (int i = 0; i < n; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-15) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

// integral of exp(-V / kT) over [u, v], split at the spline's knots (smooth pieces)
double boltzmann_integral(double u, double v, double a0, double a1, double h, double d, double kw, double kT) {
    static const GaussLegendre gl;
    const double m = 0.5 * (a0 + a1);
    double cuts[6] = {u, a0, m, a1, v, v};
    double s = 0.0;
    double prev = u;
    for (int c = 1; c < 5; ++c) {
        const double next = std::min(std::max(cuts[c], u), v);
        if (next > prev) {
            const double half = 0.5 * (next - prev), mid = 0.5 * (next + prev);
            for (int i = 0; i < 64; ++i)
                s += half * gl.w[i] * std::exp(-dw_value(mid + half * gl.x[i], a0, a1, h, d, kw) / kT);
            prev = next;
        }
    }
    return s;
}

}  // namespace

extern "C" fmm_status fmm_lambda_pfc(double pH, double pKa_ref, double barrier, double kT, double a0, double a1,
                                     double kwall, double lo, double hi, double* delta) {
    const double m = 0.5 * (a0 + a1);
    if (!delta || !(kT > 0.0) || !(a0 < a1) || !(lo < m) || !(hi > m) || !(kwall >= 0.0)) return FMM_ERR_ARG;
    const double target = std::log(10.0) * (pH - pKa_ref);
    const double zp = boltzmann_integral(lo, m, a0, a1, barrier, 0.0, kwall, kT);  // independent of delta
    // ln(Z_deprot / Z_prot) decreases monotonically in delta: bisect
    auto g = [&](double d) { return std::log(boltzmann_integral(m, hi, a0, a1, barrier, d, kwall, kT) / zp) - target; };
    double dl = -(60.0 + std::fabs(target)) * kT, dh = (60.0 + std::fabs(target)) * kT;
    for (int it = 0; it < 200 && dh - dl > 1e-14 * (1.0 + std::fabs(dl)); ++it) {
        const double mid = 0.5 * (dl + dh);
        if (g(mid) > 0.0) dl = mid;
        else dh = mid;
    }
    *delta = 0.5 * (dl + dh);
    return FMM_OK;
}
