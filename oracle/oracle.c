/*
 * Oracle for the FMM constant-pH electrostatics path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct FP64 CPU code.  It computes the exact
 * quantities that the GPU fast multipole method approximates:
 *
 *   q_i      = qA_i + lambda_{s(i)} (qB_i - qA_i)            (Sec. 2.1, Eq. 1:
 *              the Hamiltonian is linear in lambda and the forms differ only
 *              in their charges; read as charge interpolation, the Hamiltonian
 *              form's intra-site difference being computed separately)
 *   phi_i    = sum_{j != i} q_j / |x_i - x_j|                 (open boundary)
 *   phi_i    = dE_Ewald/dq_i                                   (periodic cube,
 *              tinfoil boundary, uniform neutralising background)
 *   grad_i   = gradient of the potential of all other charges at x_i
 *
 * and the binning specification (Morton keys of the leaf cells, a stable
 * sort, leaf ranges) that the GPU binning must reproduce bit for bit.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared oracle.c -lm
 * (-ffp-contract=off: the binning spec forbids fused multiply-add.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- charges (Sec. 2.1, Eq. 1 with charge-only differences between forms) ---- */
void orc_charges(int n, const float* qA, const float* qB, const int32_t* site,
                 int n_sites, const float* lam, double* q, double* dq) {
    for (int i = 0; i < n; ++i) {
        double a = qA[i], b = qB[i];
        int s = site[i];
        if (s >= 0 && s < n_sites) {
            double l = lam[s];
            q[i] = a + l * (b - a);
            dq[i] = b - a;
        } else {
            q[i] = a;
            dq[i] = 0.0;
        }
    }
}

/* ---- open boundary: direct Coulomb sum, every pair i != j ---- */
void orc_direct(int n, const double* x, const double* q, int nt, const int32_t* tgt,
                double* phi, double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t) {
        int i = tgt ? tgt[t] : t;
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[3 * i] - x[3 * j];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double ir = 1.0 / r;
            p += q[j] * ir;
            double ir3 = q[j] * ir * ir * ir;
            /* gradient of q_j/|x - x_j| with respect to x */
            gx -= ir3 * dx;
            gy -= ir3 * dy;
            gz -= ir3 * dz;
        }
        phi[t] = p;
        grad[3 * t] = gx;
        grad[3 * t + 1] = gy;
        grad[3 * t + 2] = gz;
    }
}

/* ---- periodic cube: classical Ewald sum ----
 * E = 1/2 sum_i sum_j sum'_n q_i q_j erfc(a r)/r
 *   + (2 pi / V) sum_{k != 0} exp(-k^2 / 4a^2) / k^2 |S(k)|^2
 *   - (a / sqrt(pi)) sum_i q_i^2 - pi Q^2 / (2 V a^2)
 * with S(k) = sum_j q_j exp(i k.x_j), Q = sum q, k = 2 pi m / L.
 * The prime drops j == i in the n = 0 image.  phi_i = dE/dq_i. */

/* Reciprocal-space structure factors for the half space of m vectors
 * (m_x > 0, or m_x == 0 and m_y > 0, or m_x == m_y == 0 and m_z > 0). */
static int half_space(int mx, int my, int mz) {
    if (mx > 0) return 1;
    if (mx < 0) return 0;
    if (my > 0) return 1;
    if (my < 0) return 0;
    return mz > 0;
}

/* Wall-clock seconds of the two phases of the last orc_ewald call (structure factors; the
 * per-target sums), for timing the oracle as a CPU baseline.  Timing only: it changes nothing
 * that is computed. */
static double g_ewald_phase_s[2];
extern double omp_get_wtime(void);
void orc_ewald_phase_seconds(double* out) {
    out[0] = g_ewald_phase_s[0];
    out[1] = g_ewald_phase_s[1];
}

void orc_ewald(int n, const double* x, const double* q, double L, double alpha,
               double rc, int mmax, int nt, const int32_t* tgt, double* phi,
               double* grad) {
    const double t_start = omp_get_wtime();
    const double V = L * L * L;
    const int side = 2 * mmax + 1;
    /* enumerate k vectors */
    int nk = 0;
    for (int mx = -mmax; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz)
                if (half_space(mx, my, mz) && mx * mx + my * my + mz * mz <= mmax * mmax) ++nk;
    int* km = (int*)malloc(sizeof(int) * 3 * (nk > 0 ? nk : 1));
    double* kw = (double*)malloc(sizeof(double) * (nk > 0 ? nk : 1));
    double* Sre = (double*)calloc(nk > 0 ? nk : 1, sizeof(double));
    double* Sim = (double*)calloc(nk > 0 ? nk : 1, sizeof(double));
    nk = 0;
    for (int mx = -mmax; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz)
                if (half_space(mx, my, mz) && mx * mx + my * my + mz * mz <= mmax * mmax) {
                    km[3 * nk] = mx; km[3 * nk + 1] = my; km[3 * nk + 2] = mz;
                    double k2 = (2 * M_PI / L) * (2 * M_PI / L) * (double)(mx * mx + my * my + mz * mz);
                    /* factor 2 for the omitted -k half */
                    kw[nk] = 2.0 * (4.0 * M_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
                    ++nk;
                }
    (void)side;
    /* S(k) = sum_j q_j exp(i k.x_j), threads own disjoint k ranges */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nk; ++k) {
        double kx = 2 * M_PI / L * km[3 * k], ky = 2 * M_PI / L * km[3 * k + 1],
               kz = 2 * M_PI / L * km[3 * k + 2];
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            double ph = kx * x[3 * j] + ky * x[3 * j + 1] + kz * x[3 * j + 2];
            sr += q[j] * cos(ph);
            si += q[j] * sin(ph);
        }
        Sre[k] = sr;
        Sim[k] = si;
    }
    double Q = 0.0;
    for (int j = 0; j < n; ++j) Q += q[j];
    const double t_sf = omp_get_wtime();
    const double rc2 = rc * rc;
    const double two_a_sqrtpi = 2.0 * alpha / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 8)
    for (int t = 0; t < nt; ++t) {
        int i = tgt ? tgt[t] : t;
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        /* real space: all images within rc */
        for (int j = 0; j < n; ++j) {
            double d0[3];
            for (int a = 0; a < 3; ++a) {
                double d = x[3 * i + a] - x[3 * j + a];
                d0[a] = d - L * floor(d / L + 0.5); /* minimum image */
            }
            int lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                lo[a] = (int)ceil((-rc - d0[a]) / L);
                hi[a] = (int)floor((rc - d0[a]) / L);
            }
            for (int nx = lo[0]; nx <= hi[0]; ++nx)
                for (int ny = lo[1]; ny <= hi[1]; ++ny)
                    for (int nz = lo[2]; nz <= hi[2]; ++nz) {
                        double dx = d0[0] + nx * L, dy = d0[1] + ny * L, dz = d0[2] + nz * L;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > rc2) continue;
                        if (j == i && r2 == 0.0) continue; /* self, zero image */
                        double r = sqrt(r2);
                        double e = erfc(alpha * r) / r;
                        p += q[j] * e;
                        double f = q[j] * (e + two_a_sqrtpi * exp(-alpha * alpha * r2)) / r2;
                        gx -= f * dx;
                        gy -= f * dy;
                        gz -= f * dz;
                    }
        }
        /* reciprocal space */
        for (int k = 0; k < nk; ++k) {
            double kx = 2 * M_PI / L * km[3 * k], ky = 2 * M_PI / L * km[3 * k + 1],
                   kz = 2 * M_PI / L * km[3 * k + 2];
            double ph = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            double c = cos(ph), s = sin(ph);
            /* Re(exp(-i k.x) S) and its gradient in x */
            double re = c * Sre[k] + s * Sim[k];
            double dre = -s * Sre[k] + c * Sim[k]; /* d/dph of re */
            p += kw[k] * re;
            gx += kw[k] * dre * kx;
            gy += kw[k] * dre * ky;
            gz += kw[k] * dre * kz;
        }
        p -= two_a_sqrtpi * q[i];
        p -= M_PI * Q / (V * alpha * alpha);
        phi[t] = p;
        grad[3 * t] = gx;
        grad[3 * t + 1] = gy;
        grad[3 * t + 2] = gz;
    }
    g_ewald_phase_s[0] = t_sf - t_start;
    g_ewald_phase_s[1] = omp_get_wtime() - t_sf;
    free(km);
    free(kw);
    free(Sre);
    free(Sim);
}

/* ---- Ewald pair potential (for the Hamiltonian-interpolation correction) ----
 * psi(r): potential at displacement r of a unit charge and all its periodic
 * images in a cube of edge L, tinfoil boundary, uniform neutralising
 * background (the pair potential of the Ewald energy above):
 *   psi(r) = sum_n erfc(alpha |r + nL|) / |r + nL|
 *          + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 cos(k . r)
 *          - pi / (V alpha^2).
 * With self != 0 the result is the self-image term psi_0 = lim_{r -> 0}
 * (psi(r) - 1/|r|): the n = 0 real-space term is replaced by its limit
 * -2 alpha / sqrt(pi) (r is then ignored).  grad = d psi / d r (zero for
 * self).  Images within rc, reciprocal indices |m| <= mmax. */
void orc_ewald_pair(const double* r, int self, double L, double alpha, double rc, int mmax, double* psi,
                    double* grad) {
    const double V = L * L * L;
    double d0[3] = {0.0, 0.0, 0.0};
    if (!self)
        for (int a = 0; a < 3; ++a) d0[a] = r[a];
    double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)ceil((-rc - d0[a]) / L) - 1;
        hi[a] = (int)floor((rc - d0[a]) / L) + 1;
    }
    for (int nx = lo[0]; nx <= hi[0]; ++nx)
        for (int ny = lo[1]; ny <= hi[1]; ++ny)
            for (int nz = lo[2]; nz <= hi[2]; ++nz) {
                const double dx = d0[0] + nx * L, dy = d0[1] + ny * L, dz = d0[2] + nz * L;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > rc * rc) continue;
                if (self && nx == 0 && ny == 0 && nz == 0) continue;
                const double rn = sqrt(r2);
                const double e = erfc(alpha * rn) / rn;
                p += e;
                const double f = (e + 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * r2)) / r2;
                gx -= f * dx;
                gy -= f * dy;
                gz -= f * dz;
            }
    if (self) p -= 2.0 * alpha / sqrt(M_PI);
    for (int mx = -mmax; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz) {
                const int m2 = mx * mx + my * my + mz * mz;
                if (m2 == 0 || m2 > mmax * mmax) continue;
                const double kx = 2.0 * M_PI / L * mx, ky = 2.0 * M_PI / L * my, kz = 2.0 * M_PI / L * mz;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double w = 4.0 * M_PI / V * exp(-k2 / (4.0 * alpha * alpha)) / k2;
                const double ph = kx * d0[0] + ky * d0[1] + kz * d0[2];
                p += w * cos(ph);
                const double sw = -w * sin(ph);
                gx += sw * kx;
                gy += sw * ky;
                gz += sw * kz;
            }
    p -= M_PI / (V * alpha * alpha);
    *psi = p;
    grad[0] = self ? 0.0 : gx;
    grad[1] = self ? 0.0 : gy;
    grad[2] = self ? 0.0 : gz;
}

/* ---- binning specification ----
 * Per axis: u = (double)x - origin; periodic: u -= L*floor(u/L), then u
 * outside [0, L) is folded to 0; open: u outside [0, L] flags the domain
 * error bit.  Cell index i = floor(u * (2^d / L)) in FP64 without FMA,
 * clamped to [0, 2^d - 1].  Morton key: bit 3b = i_x bit b, 3b+1 = i_y bit b,
 * 3b+2 = i_z bit b.  The permutation is the stable sort of atoms by key
 * (ties broken by the original index).  start/count per leaf key, empty
 * leaves start at their insertion point.  status bit 1 = atom outside an
 * open box. */
void orc_bin(int n, const float* x, const double* origin, double L, int depth,
             int periodic, uint32_t* key, uint32_t* perm, uint32_t* start,
             uint32_t* count, int32_t* status) {
    const int nb = 1 << depth;
    const double s = ldexp(1.0, depth) / L;
    const long nleaf = 1L << (3 * depth);
    int st = 0;
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double u = (double)x[3 * i + a] - origin[a];
            if (periodic) {
                u = u - L * floor(u / L);
                if (u < 0.0 || u >= L) u = 0.0;
            } else if (!(u >= 0.0 && u <= L)) {
                st |= 1;
            }
            double f = floor(u * s);
            int ci;
            if (!(f >= 0.0)) ci = 0;
            else if (f > (double)(nb - 1)) ci = nb - 1;
            else ci = (int)f;
            c[a] = ci;
        }
        uint32_t k = 0;
        for (int b = 0; b < depth; ++b) {
            k |= (uint32_t)((c[0] >> b) & 1) << (3 * b);
            k |= (uint32_t)((c[1] >> b) & 1) << (3 * b + 1);
            k |= (uint32_t)((c[2] >> b) & 1) << (3 * b + 2);
        }
        key[i] = k;
    }
    /* counting sort: stable because atoms are visited in index order */
    memset(count, 0, sizeof(uint32_t) * nleaf);
    for (int i = 0; i < n; ++i) count[key[i]]++;
    uint32_t acc = 0;
    for (long b = 0; b < nleaf; ++b) {
        start[b] = acc;
        acc += count[b];
    }
    uint32_t* fill = (uint32_t*)malloc(sizeof(uint32_t) * nleaf);
    memcpy(fill, start, sizeof(uint32_t) * nleaf);
    for (int i = 0; i < n; ++i) perm[fill[key[i]]++] = (uint32_t)i;
    free(fill);
    *status = st;
}

int orc_nthreads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
