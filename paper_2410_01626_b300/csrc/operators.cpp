// Host-side (FP64) construction of the fast multipole translation operators.
//
// Solid harmonics.  With the generating function
//     G(r; s, t) = exp( s z + (s t / 2)(x - i y) - (s / (2t))(x + i y) ),
// the regular solid harmonics R_n^m (|m| <= n) are the coefficients of
// s^n t^m.  The exponent's vector is null, so every R_n^m is harmonic, and
// G(a + b) = G(a) G(b) gives the addition theorem
//     R_n^m(a + b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b).
// In spherical coordinates R_n^m = r^n P_n^|m|(cos th) e^{-i m ph} / (n+|m|)!
// (times (-1)^m for m < 0).  The irregular harmonics
//     I_n^m = (n-|m|)! P_n^|m|(cos th) e^{-i m ph} / r^{n+1}  (same sign rule)
// satisfy 1/|r - v| = sum_{n,m} conj(R_n^m(v)) I_n^m(r) for |v| < |r|
// (Legendre addition theorem).  Both obey C_n^{-m} = (-1)^m conj(C_n^m).
//
// Fast multipole method (Greengard and Rokhlin; the paper's FMM, Sec. 2.6):
//   multipole about a:   phi(r) = sum M_n^m I_n^m(r - a),  M_n^m = sum q conj(R_n^m(v - a))
//   local about b:       phi(r) = sum L_n^m R_n^m(r - b)
//   M2M (a -> b):        M_n^m(b) = sum_{k,l} conj(R_{n-k}^{m-l}(a - b)) M_k^l(a)
//   L2L (a -> b):        L_k^l(b) = sum_{n>=k,m} L_n^m(a) R_{n-k}^{m-l}(b - a)
//   M2L (source a, target b, t = b - a):
//                        L_k^l = (-1)^{k+l} sum_{n,m} M_n^m I_{n+k}^{m-l}(t)
//
// Stored coefficients are normalised and scaled per level so that every
// operator is level independent and of order one (Schmidt normalisation):
//   Mhat_n^m = M_n^m N_n^m / h^n,   Lhat_n^m = L_n^m h^{n+1} / N_n^m,
//   N_n^m = sqrt((n+m)!(n-m)!),  h = box edge of the level.
// Real form: a symmetric complex vector is stored as (p+1)^2 reals, degree n
// at offsets n^2 .. n^2+2n: [Re C_n^0, Re C_n^1, Im C_n^1, ..., Re C_n^n, Im C_n^n].
//
// Periodic boundary (tinfoil Ewald convention with a neutralising
// background): the pair potential psi(r) of a unit cube lattice splits, for
// |r| < 2, into the 27 nearest images, a quadratic background term and a
// harmonic remainder,
//     psi(r) = sum_{n in {-1,0,1}^3} 1/|r - n| + (2 pi / 3V)|r|^2 + h(r),
// because lap psi = -4 pi sum delta + 4 pi / V.  The tree handles the 27
// images (levels >= 1 use periodic neighbour and interaction lists), the
// quadratic term is applied per atom from the total charge Q, dipole D and
// trace T = sum q |u|^2, and h = sum g_l^m R_l^m becomes the root-level
// lattice operator  L_k^k' = sum_{n,m'} (-1)^{n+m'} g_{n+k}^{k'-m'} M_n^m'.
// The coefficients g are obtained by projecting h, evaluated with an FP64
// Ewald sum on a sphere of radius 1/2, onto the harmonics with an exact
// Gauss-Legendre x trapezoid quadrature.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "operators.h"

namespace fmmcph {

using cd = std::complex<double>;

static inline int cidx(int n, int m) { return n * n + n + m; }  // complex index, m in [-n, n]

static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

double norm_nm(int n, int m) {
    if (m < 0) m = -m;
    return std::sqrt(fact(n + m) * fact(n - m));
}

static void fill_negative(std::vector<cd>& C, int P) {
    for (int n = 0; n <= P; ++n)
        for (int m = 1; m <= n; ++m)
            C[cidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(C[cidx(n, m)]);
}

void regular_c(const double u[3], int P, std::vector<cd>& R) {
    R.assign((P + 1) * (P + 1), cd(0, 0));
    const double x = u[0], y = u[1], z = u[2];
    const double r2 = x * x + y * y + z * z;
    const cd w(x, -y);
    R[cidx(0, 0)] = 1.0;
    for (int m = 0; m <= P; ++m) {
        if (m > 0) R[cidx(m, m)] = R[cidx(m - 1, m - 1)] * w / (2.0 * m);
        for (int n = m + 1; n <= P; ++n) {
            cd a = R[cidx(n - 1, m)];
            cd b = (n - 2 >= m) ? R[cidx(n - 2, m)] : cd(0, 0);
            R[cidx(n, m)] = ((2.0 * n - 1.0) * z * a - r2 * b) / double((n + m) * (n - m));
        }
    }
    fill_negative(R, P);
}

void irregular_c(const double t[3], int P, std::vector<cd>& I) {
    I.assign((P + 1) * (P + 1), cd(0, 0));
    const double x = t[0], y = t[1], z = t[2];
    const double r2 = x * x + y * y + z * z;
    const cd w(x, -y);
    I[cidx(0, 0)] = 1.0 / std::sqrt(r2);
    for (int m = 0; m <= P; ++m) {
        if (m > 0) I[cidx(m, m)] = I[cidx(m - 1, m - 1)] * (2.0 * m - 1.0) * w / r2;
        for (int n = m + 1; n <= P; ++n) {
            cd a = I[cidx(n - 1, m)];
            cd b = (n - 2 >= m) ? I[cidx(n - 2, m)] : cd(0, 0);
            I[cidx(n, m)] = ((2.0 * n - 1.0) * z * a - double((n + m - 1) * (n - m - 1)) * b) / r2;
        }
    }
    fill_negative(I, P);
}

// Real-form matrix of a complex-linear map given entry-wise by coef(k,l,n,m)
// (output degree/order k,l; input n,m; signed orders), with row scale
// rs(k,l) and column scale cs(n,m) (applied to the complex entries).
template <class Coef, class RS, class CS>
static void build_real(int P, Coef coef, RS rs, CS cs, double* out) {
    const int nc = (P + 1) * (P + 1);
    std::memset(out, 0, sizeof(double) * nc * nc);
    for (int k = 0; k <= P; ++k)
        for (int l = 0; l <= k; ++l) {
            const double r = rs(k, l);
            for (int n = 0; n <= P; ++n)
                for (int m = 0; m <= n; ++m) {
                    const double c = cs(n, m);
                    // d L_k^l / d (Re M_n^m) and d / d (Im M_n^m)
                    cd dre, dim;
                    if (m == 0) {
                        dre = coef(k, l, n, 0);
                        dim = 0.0;
                    } else {
                        const double sg = (m & 1) ? -1.0 : 1.0;
                        cd a = coef(k, l, n, m), b = coef(k, l, n, -m);
                        dre = a + sg * b;
                        dim = cd(0, 1) * a - cd(0, 1) * sg * b;
                    }
                    dre *= r * c;
                    dim *= r * c;
                    const int col_re = (m == 0) ? n * n : n * n + 2 * m - 1;
                    const int row_re = (l == 0) ? k * k : k * k + 2 * l - 1;
                    out[row_re * nc + col_re] = dre.real();
                    if (m > 0) out[row_re * nc + col_re + 1] = dim.real();
                    if (l > 0) {
                        out[(row_re + 1) * nc + col_re] = dre.imag();
                        if (m > 0) out[(row_re + 1) * nc + col_re + 1] = dim.imag();
                    }
                }
        }
}

void op_m2l(int P, const int o[3], double* out) {
    // source box = target box + o (in units of the level's box edge); t = target - source
    const double t[3] = {-double(o[0]), -double(o[1]), -double(o[2])};
    std::vector<cd> I;
    irregular_c(t, 2 * P, I);
    auto coef = [&](int k, int l, int n, int m) -> cd {
        int mm = m - l;
        if (mm < -(n + k) || mm > n + k) return 0.0;
        return (((k + l) & 1) ? -1.0 : 1.0) * I[cidx(n + k, mm)];
    };
    build_real(P, coef, [](int k, int l) { return 1.0 / norm_nm(k, l); },
               [](int n, int m) { return 1.0 / norm_nm(n, m); }, out);
}

void op_m2m(int P, int oct, double* out) {
    // child centre - parent centre, in units of the child edge
    const double d[3] = {(oct & 1) - 0.5, ((oct >> 1) & 1) - 0.5, ((oct >> 2) & 1) - 0.5};
    std::vector<cd> R;
    regular_c(d, P, R);
    auto coef = [&](int n, int m, int k, int l) -> cd {  // out (n,m), in (k,l)
        if (k > n) return 0.0;
        int mm = m - l;
        if (mm < -(n - k) || mm > n - k) return 0.0;
        return std::conj(R[cidx(n - k, mm)]);
    };
    build_real(P, coef, [](int n, int m) { return norm_nm(n, m) / std::ldexp(1.0, n); },
               [](int k, int l) { return 1.0 / norm_nm(k, l); }, out);
}

void op_l2l(int P, int oct, double* out) {
    const double d[3] = {(oct & 1) - 0.5, ((oct >> 1) & 1) - 0.5, ((oct >> 2) & 1) - 0.5};
    std::vector<cd> R;
    regular_c(d, P, R);
    auto coef = [&](int k, int l, int n, int m) -> cd {
        if (n < k) return 0.0;
        int mm = m - l;
        if (mm < -(n - k) || mm > n - k) return 0.0;
        return R[cidx(n - k, mm)];
    };
    build_real(P, coef, [](int k, int l) { return 1.0 / norm_nm(k, l); },
               [](int n, int m) { return norm_nm(n, m) / std::ldexp(1.0, n + 1); }, out);
}

// ---- periodic lattice ----

// psi(r) - 1/|r| for the unit cube (V = 1): Ewald sum, tinfoil, neutralising background.
static double ewald_psi_minus_coulomb(const double r[3]) {
    const double alpha = 5.0;
    const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double s = -std::erf(alpha * rn) / rn;
    for (int a = -2; a <= 2; ++a)
        for (int b = -2; b <= 2; ++b)
            for (int c = -2; c <= 2; ++c) {
                if (!a && !b && !c) continue;
                double dx = r[0] + a, dy = r[1] + b, dz = r[2] + c;
                double d = std::sqrt(dx * dx + dy * dy + dz * dz);
                s += std::erfc(alpha * d) / d;
            }
    const int mmax = 10;
    const double tp = 2.0 * M_PI;
    // cos(k.r) via products of per-axis phases; sum over the half space x2
    std::vector<cd> ex(2 * mmax + 1), ey(2 * mmax + 1), ez(2 * mmax + 1);
    for (int m = -mmax; m <= mmax; ++m) {
        ex[m + mmax] = std::polar(1.0, tp * m * r[0]);
        ey[m + mmax] = std::polar(1.0, tp * m * r[1]);
        ez[m + mmax] = std::polar(1.0, tp * m * r[2]);
    }
    double rec = 0.0;
    for (int a = -mmax; a <= mmax; ++a)
        for (int b = -mmax; b <= mmax; ++b)
            for (int c = -mmax; c <= mmax; ++c) {
                int m2 = a * a + b * b + c * c;
                if (m2 == 0 || m2 > mmax * mmax) continue;
                double k2 = tp * tp * m2;
                double w = 4.0 * M_PI * std::exp(-k2 / (4.0 * alpha * alpha)) / k2;
                rec += w * (ex[a + mmax] * ey[b + mmax] * ez[c + mmax]).real();
            }
    s += rec;
    s -= M_PI / (alpha * alpha);
    return s;
}

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // final derivative for the weight
                p0 = 1.0;
                p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[i] = z;
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Complex symmetric coefficients g_l^m (un-normalised) of the harmonic
// remainder h, degrees 0..Q, for the unit cube.
void lattice_coefficients(int Q, std::vector<std::complex<double>>& g) {
    const int nth = 48, nph = 96;
    const double rho = 0.5;
    std::vector<double> xg, wg;
    gauss_legendre(nth, xg, wg);
    const int nreal = (Q + 1) * (Q + 1);
    std::vector<double> num(nreal, 0.0), den(nreal, 0.0);
    std::vector<cd> R;
    for (int i = 0; i < nth; ++i) {
        const double ct = xg[i], st = std::sqrt(1.0 - ct * ct);
        for (int j = 0; j < nph; ++j) {
            const double ph = 2.0 * M_PI * j / nph;
            const double r[3] = {rho * st * std::cos(ph), rho * st * std::sin(ph), rho * ct};
            double hv = ewald_psi_minus_coulomb(r);
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b)
                    for (int c = -1; c <= 1; ++c) {
                        if (!a && !b && !c) continue;
                        double dx = r[0] - a, dy = r[1] - b, dz = r[2] - c;
                        hv -= 1.0 / std::sqrt(dx * dx + dy * dy + dz * dz);
                    }
            hv -= (2.0 * M_PI / 3.0) * rho * rho;
            const double w = wg[i] * 2.0 * M_PI / nph;
            regular_c(r, Q, R);
            for (int n = 0; n <= Q; ++n)
                for (int m = 0; m <= n; ++m) {
                    // h = sum_n [ghat_n^0 Rh_n^0 + 2 sum_m (Re ghat Re Rh - Im ghat Im Rh)]
                    const double Nn = norm_nm(n, m);
                    const cd Rh = R[cidx(n, m)] * Nn;
                    if (m == 0) {
                        num[n * n] += w * Rh.real() * hv;
                        den[n * n] += w * Rh.real() * Rh.real();
                    } else {
                        const double cr = 2.0 * Rh.real(), ci = -2.0 * Rh.imag();
                        num[n * n + 2 * m - 1] += w * cr * hv;
                        den[n * n + 2 * m - 1] += w * cr * cr;
                        num[n * n + 2 * m] += w * ci * hv;
                        den[n * n + 2 * m] += w * ci * ci;
                    }
                }
        }
    }
    g.assign((Q + 1) * (Q + 1), cd(0, 0));
    for (int n = 0; n <= Q; ++n)
        for (int m = 0; m <= n; ++m) {
            const double Nn = norm_nm(n, m);
            cd gh;
            if (m == 0) gh = num[n * n] / den[n * n];
            else gh = cd(num[n * n + 2 * m - 1] / den[n * n + 2 * m - 1], num[n * n + 2 * m] / den[n * n + 2 * m]);
            g[cidx(n, m)] = gh * Nn;  // un-normalised: h = sum g R
        }
    // symmetric completion; odd degrees and degree 2 vanish by cubic symmetry
    for (int n = 0; n <= Q; ++n) {
        if ((n & 1) || n == 2)
            for (int m = 0; m <= n; ++m) g[cidx(n, m)] = 0.0;
        for (int m = 1; m <= n; ++m) g[cidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(g[cidx(n, m)]);
    }
}

void op_lattice(int P, double* out) {
    std::vector<cd> g;
    lattice_coefficients(2 * P, g);
    auto coef = [&](int k, int kap, int n, int mu) -> cd {
        int mm = kap - mu;
        if (mm < -(n + k) || mm > n + k) return 0.0;
        return (((n + mu) & 1) ? -1.0 : 1.0) * g[cidx(n + k, mm)];
    };
    build_real(P, coef, [](int k, int l) { return 1.0 / norm_nm(k, l); },
               [](int n, int m) { return 1.0 / norm_nm(n, m); }, out);
}

void regular_real_hat(int P, const double u[3], double* out) {
    std::vector<cd> R;
    regular_c(u, P, R);
    for (int n = 0; n <= P; ++n) {
        out[n * n] = R[cidx(n, 0)].real() * norm_nm(n, 0);
        for (int m = 1; m <= n; ++m) {
            cd v = R[cidx(n, m)] * norm_nm(n, m);
            out[n * n + 2 * m - 1] = v.real();
            out[n * n + 2 * m] = v.imag();
        }
    }
}

}  // namespace fmmcph
