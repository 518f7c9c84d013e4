// Host-side FP64 tables of the plan: window Fourier coefficients, kernel
// Fourier coefficients b_l (Eq. K_RF and the footnote to Sec. 4), the
// regulariser of the ball domain, the coefficient-slot multiplier and the
// real trigonometric transform matrices; plus a small dense symmetric
// eigensolver for the Lanczos projection.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ml_internal.h"

namespace ml {

static const double kPi = 3.14159265358979323846;

// I_0(x) = sum_k (x/2)^{2k} / (k!)^2 (Abramowitz & Stegun 9.6.12); all terms
// are positive, so the partial sums converge monotonically in FP64.
double bessel_i0(double x)
{
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// The Kaiser-Bessel pair used by the NFFT (window phi with shape
// b = pi (2 - 1/sigma_os)) with half-width h (in grid cells; h = W/2 for a
// window of W taps, any real h > 0):  phi(x) = (1/pi) sinh(b sqrt(h^2 - n^2 x^2)) /
// sqrt(h^2 - n^2 x^2) on |x| <= h/n, with Fourier transform
// phi_hat(k) = (1/n) I_0(h sqrt(b^2 - (2 pi k / n)^2)) for |k| <= n(1 - 1/(2 sigma_os)).
// The device evaluates the normalised window phi_n = pi h / sinh(b h) * phi
// (phi_n(0) = 1), so its coefficients carry the same factor.
void window_fourier(int n_os, double h, double b, int kmax, std::vector<double> &out)
{
    out.assign(kmax + 1, 0.0);
    const double c = kPi * h / std::sinh(b * h);
    for (int k = 0; k <= kmax; ++k) {
        const double w = 2.0 * kPi * k / n_os;
        const double arg = b * b - w * w;
        out[k] = arg > 0 ? c * bessel_i0(h * std::sqrt(arg)) / n_os : 0.0;
    }
}

// Physicists' Hermite recursion for the derivatives of exp(-r^2/s^2):
// d^k/dr^k = (-1)^k s^{-k} H_k(r/s) exp(-(r/s)^2).
static void gauss_derivs(double r, double s, int p, std::vector<double> &dk)
{
    const double z = r / s;
    std::vector<double> H(p + 1);
    H[0] = 1.0;
    if (p >= 1) H[1] = 2.0 * z;
    for (int k = 1; k < p; ++k) H[k + 1] = 2.0 * z * H[k] - 2.0 * k * H[k - 1];
    const double e = std::exp(-z * z);
    dk.assign(p, 0.0);
    for (int k = 0; k < p; ++k) dk[k] = ((k & 1) ? -1.0 : 1.0) * std::pow(s, -k) * H[k] * e;
}

// Derivatives of the Laplacian exp(-r/s): d^k/dr^k = (-1/s)^k exp(-r/s).
static void laplace_derivs(double r, double s, int p, std::vector<double> &dk)
{
    const double e = std::exp(-r / s);
    dk.assign(p, 0.0);
    double f = 1.0;
    for (int k = 0; k < p; ++k) {
        dk[k] = f * e;
        f *= -1.0 / s;
    }
}

// Solve A x = rhs (n x n, row-major) by Gaussian elimination with partial pivoting.
static bool solve_dense(int n, std::vector<double> A, std::vector<double> &x)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * (n + 1) + c]) > std::fabs(A[piv * (n + 1) + c])) piv = r;
        if (A[piv * (n + 1) + c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j <= n; ++j) std::swap(A[c * (n + 1) + j], A[piv * (n + 1) + j]);
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
            for (int j = c; j <= n; ++j) A[r * (n + 1) + j] -= f * A[c * (n + 1) + j];
        }
    }
    x.assign(n, 0.0);
    for (int r = n - 1; r >= 0; --r) {
        double s = A[r * (n + 1) + n];
        for (int j = r + 1; j < n; ++j) s -= A[r * (n + 1) + j] * x[j];
        x[r] = s / A[r * (n + 1) + r];
    }
    return true;
}

// Regulariser of the ball domain: on t = (r - r_I)/eps_B in [0, 1], a
// polynomial of degree 2p-1 whose derivatives 0..p-1 at t = 0 equal those of
// the kernel (Gaussian or Laplacian) at r_I = 1/2 - eps_B (chain rule factor
// eps_B^k), whose value at t = 1 is K(1/2) and whose derivatives 1..p-1
// vanish at t = 1.
bool regulariser_coeffs(double s, double eps_B, int p, std::vector<double> &q, int kernel)
{
    const int n = 2 * p;
    const double rI = 0.5 - eps_B;
    std::vector<double> dK;
    if (kernel == ML_KERNEL_LAPLACE) laplace_derivs(rI, s, p, dK);
    else gauss_derivs(rI, s, p, dK);
    const double k_half = kernel == ML_KERNEL_LAPLACE ? std::exp(-0.5 / s) : std::exp(-0.25 / (s * s));
    std::vector<double> A((size_t)n * (n + 1), 0.0);
    for (int k = 0; k < p; ++k) {
        for (int j = k; j < n; ++j) {
            double f = 1.0;  // j!/(j-k)!
            for (int i = 0; i < k; ++i) f *= (double)(j - i);
            A[k * (n + 1) + j] = (j == k) ? f : 0.0;        // at t = 0 only t^k survives
            A[(p + k) * (n + 1) + j] = f;                    // at t = 1
        }
        A[k * (n + 1) + n] = dK[k] * std::pow(eps_B, k);
        A[(p + k) * (n + 1) + n] = (k == 0) ? k_half : 0.0;
    }
    return solve_dense(n, A, q);
}

// Inner regulariser of the Laplacian: P(r) = sum_{j<p} c_j r^{2j} with
// P^{(k)}(eps_I) = K^{(k)}(eps_I), k = 0..p-1; the k-th derivative of r^{2j}
// is (2j)!/(2j-k)! r^{2j-k}.  An even polynomial, hence smooth at the origin
// in every dimension.
bool inner_coeffs(double s, double eps_I, int p, std::vector<double> &c)
{
    std::vector<double> dK;
    laplace_derivs(eps_I, s, p, dK);
    std::vector<double> A((size_t)p * (p + 1), 0.0);
    for (int k = 0; k < p; ++k) {
        for (int j = 0; j < p; ++j) {
            const int e = 2 * j;
            if (e < k) continue;
            double f = 1.0;
            for (int i = 0; i < k; ++i) f *= (double)(e - i);
            A[k * (p + 1) + j] = f * std::pow(eps_I, e - k);
        }
        A[k * (p + 1) + p] = dK[k];
    }
    return solve_dense(p, A, c);
}

// The Laplacian's K_R at distance r (ball domain): the inner polynomial on
// r < eps_I, the kernel up to 1/2 - eps_B, the two-point Taylor regulariser on
// (1/2 - eps_B, 1/2] and its end value beyond.
double laplace_regularised(double r, const LaplaceReg &g)
{
    if (r < g.eps_I) {
        const double r2 = r * r;
        double v = 0.0;
        for (int j = (int)g.c.size() - 1; j >= 0; --j) v = v * r2 + g.c[j];
        return v;
    }
    if (r <= 0.5 - g.eps_B) return std::exp(-r / g.s);
    double t = (r - (0.5 - g.eps_B)) / g.eps_B;
    if (t > 1.0) t = 1.0;
    double v = 0.0;
    for (int j = (int)g.q.size() - 1; j >= 0; --j) v = v * t + g.q[j];
    return v;
}

bool laplace_reg_init(double s, double eps_B, double eps_I, int p, LaplaceReg &g)
{
    g.s = s;
    g.eps_B = eps_B;
    g.eps_I = eps_I;
    return regulariser_coeffs(s, eps_B, p, g.q, ML_KERNEL_LAPLACE) && inner_coeffs(s, eps_I, p, g.c);
}

// Largest |K_RF(y) - K_R(y)| over probe points y with ||y|| <= 1/2 - eps_B.
// b_l is even in every l_a, so the real trigonometric polynomial folds onto
// l_a = 0..N/2 with factors 1, 2, ..., 2, 1 (the half weight of the unpaired
// edge frequency counted on both sides) and cosines:
//   K_RF(y) = sum_{kappa} b_kappa prod_a f_a(kappa_a) cos(2 pi kappa_a y_a).
// Probes: radii spread over [0, 1/2 - eps_B] (a third of them inside 2 eps_I)
// along quasi-random directions (golden-angle spiral in 2-d, Fibonacci
// sphere in 3-d).
double kernel_probe_error(const std::vector<double> &bhat, int N, int d, const LaplaceReg &g, int probes)
{
    const int H = N / 2 + 1;
    const double rmax = 0.5 - g.eps_B;
    const double golden = kPi * (3.0 - std::sqrt(5.0));
    double worst = 0.0;
    std::vector<double> f((size_t)3 * H);
    for (int k = 0; k < probes; ++k) {
        const double frac = (k + 0.5) / probes;
        double r;
        if (k % 3 == 0) r = std::min(rmax, 2.0 * g.eps_I * std::fmod(0.618034 * (k + 1), 1.0));
        else r = rmax * std::pow(std::fmod(0.754878 * (k + 1), 1.0), 1.0 / d);
        double u[3] = {1.0, 0.0, 0.0};
        if (d == 1) {
            u[0] = (k & 1) ? -1.0 : 1.0;
        } else if (d == 2) {
            u[0] = std::cos(golden * k);
            u[1] = std::sin(golden * k);
        } else {
            const double z = 1.0 - 2.0 * frac;
            const double rho = std::sqrt(std::max(0.0, 1.0 - z * z));
            u[0] = rho * std::cos(golden * k);
            u[1] = rho * std::sin(golden * k);
            u[2] = z;
        }
        for (int a = 0; a < d; ++a)
            for (int q = 0; q < H; ++q) {
                const double w = (q == 0 || q == N / 2) ? 1.0 : 2.0;
                f[(size_t)a * H + q] = w * std::cos(2.0 * kPi * q * r * u[a]);
            }
        double val = 0.0;
        if (d == 1) {
            for (int q = 0; q < H; ++q) val += bhat[q] * f[q];
        } else if (d == 2) {
            for (int q1 = 0; q1 < H; ++q1) {
                double acc = 0.0;
                for (int q0 = 0; q0 < H; ++q0) acc += bhat[(size_t)q1 * H + q0] * f[q0];
                val += acc * f[H + q1];
            }
        } else {
            for (int q2 = 0; q2 < H; ++q2) {
                double acc2 = 0.0;
                for (int q1 = 0; q1 < H; ++q1) {
                    const double *row = &bhat[((size_t)q2 * H + q1) * H];
                    double acc = 0.0;
                    for (int q0 = 0; q0 < H; ++q0) acc += row[q0] * f[q0];
                    acc2 += acc * f[H + q1];
                }
                val += acc2 * f[2 * H + q2];
            }
        }
        worst = std::max(worst, std::fabs(val - laplace_regularised(r, g)));
    }
    return worst;
}

static double kernel_regularised(double r, double s, double eps_B, const std::vector<double> &q)
{
    if (eps_B <= 0 || r <= 0.5 - eps_B) return std::exp(-r * r / (s * s));
    double t = (r - (0.5 - eps_B)) / eps_B;
    if (t > 1.0) t = 1.0;
    double v = 0.0;
    for (int j = (int)q.size() - 1; j >= 0; --j) v = v * t + q[j];
    return v;
}

// b_l = N^{-d} sum_{k in I_N} K_R(k/N) exp(-2 pi i l.k/N).  K_R is even in each
// coordinate, so b_l is real, even in each l_a, and equals the cosine sum;
// only l_a = 0..N/2 are stored (dim 0 fastest).
void kernel_fourier(double s, int N, int d, double eps_B, int p_reg, std::vector<double> &bhat)
{
    const int H = N / 2 + 1;
    std::vector<double> C((size_t)H * N);  // C[l][k + N/2] = cos(2 pi l k / N)
    for (int l = 0; l < H; ++l)
        for (int k = -N / 2; k < N / 2; ++k)
            C[(size_t)l * N + (k + N / 2)] = std::cos(2.0 * kPi * (double)l * (double)k / N);
    if (eps_B <= 0) {
        // box domain: K_R is the 1-periodisation of the Gaussian,
        // sum_r exp(-|y + r|^2/s^2), a product of 1-d periodic factors
        const int R = 2 + (int)std::ceil(8.0 * s);
        std::vector<double> b1(H, 0.0);
        for (int l = 0; l < H; ++l) {
            double acc = 0.0;
            for (int k = -N / 2; k < N / 2; ++k) {
                const double y = (double)k / N;
                double kp = 0.0;
                for (int r = -R; r <= R; ++r) kp += std::exp(-(y + r) * (y + r) / (s * s));
                acc += kp * C[(size_t)l * N + (k + N / 2)];
            }
            b1[l] = acc / N;
        }
        size_t tot = 1;
        for (int a = 0; a < d; ++a) tot *= H;
        bhat.assign(tot, 1.0);
        for (size_t idx = 0; idx < tot; ++idx) {
            size_t r = idx;
            double v = 1.0;
            for (int a = 0; a < d; ++a) {
                v *= b1[r % H];
                r /= H;
            }
            bhat[idx] = v;
        }
        return;
    }
    std::vector<double> q;
    regulariser_coeffs(s, eps_B, p_reg, q, ML_KERNEL_GAUSS);
    // samples on the full grid, then cosine sums one axis at a time
    std::vector<size_t> ext(3, 1);
    for (int a = 0; a < d; ++a) ext[a] = N;
    std::vector<double> cur(ext[0] * ext[1] * ext[2]);
    for (size_t z = 0; z < ext[2]; ++z)
        for (size_t y = 0; y < ext[1]; ++y)
            for (size_t x = 0; x < ext[0]; ++x) {
                double r2 = 0.0;
                const size_t id[3] = {x, y, z};
                for (int a = 0; a < d; ++a) {
                    const double t = ((double)id[a] - N / 2) / N;
                    r2 += t * t;
                }
                cur[(z * ext[1] + y) * ext[0] + x] = kernel_regularised(std::sqrt(r2), s, eps_B, q);
            }
    for (int a = 0; a < d; ++a) {
        std::vector<size_t> next = ext;
        next[a] = H;
        std::vector<double> out(next[0] * next[1] * next[2], 0.0);
        size_t stride = 1;
        for (int b2 = 0; b2 < a; ++b2) stride *= next[b2];
        const size_t inner = stride;
        size_t outer = 1;
        for (int b2 = a + 1; b2 < 3; ++b2) outer *= ext[b2];
        for (size_t o = 0; o < outer; ++o)
            for (size_t l = 0; l < (size_t)H; ++l)
                for (size_t i = 0; i < inner; ++i) {
                    double acc = 0.0;
                    for (size_t k = 0; k < (size_t)N; ++k)
                        acc += C[l * N + k] * cur[(o * ext[a] + k) * inner + i];
                    out[(o * H + l) * inner + i] = acc / N;
                }
        cur.swap(out);
        ext = next;
    }
    bhat.swap(cur);
}

// Multiplier over coefficient slots.  Per dim, slot s <= N/2 is the cosine of
// frequency s, slot N/2 + j (j = 1..N/2) the sine of frequency j.  The
// convolution kernel of the grid step has Fourier weights
//   w_l = b_l / (n_os^{2d} prod_a phi_hat(l_a)^2)
// on the symmetric set {-N/2..N/2}^d with half weight on each edge frequency
// (the real part of Alg. 1's sum over I_N); folding the pairs +-l gives the
// per-dim factor c(0) = 1, c(j) = 2 for 0 < j < N/2, c(N/2) = 1.
void slot_multiplier(int N, int d, int n_os, const std::vector<double> &bhat,
                     const std::vector<double> &phihat, std::vector<double> &mult)
{
    const int K = N + 1, H = N / 2 + 1;
    size_t tot = 1;
    for (int a = 0; a < d; ++a) tot *= K;
    mult.assign(tot, 0.0);
    const double scale = std::pow((double)n_os, -2.0 * d);
    for (size_t idx = 0; idx < tot; ++idx) {
        size_t r = idx, bidx = 0, bstride = 1;
        double f = scale;
        for (int a = 0; a < d; ++a) {
            const int slot = (int)(r % K);
            r /= K;
            const int kap = slot <= N / 2 ? slot : slot - N / 2;
            const double c = (kap == 0 || kap == N / 2) ? 1.0 : 2.0;
            f *= c / (phihat[kap] * phihat[kap]);
            bidx += (size_t)kap * bstride;
            bstride *= H;
        }
        mult[idx] = f * bhat[bidx];
    }
}

void trig_matrix(int N, int n_os, int s0, int L, std::vector<double> &M)
{
    const int K = N + 1;
    M.assign((size_t)K * L, 0.0);
    for (int slot = 0; slot < K; ++slot) {
        const bool is_sin = slot > N / 2;
        const int kap = is_sin ? slot - N / 2 : slot;
        for (int j = 0; j < L; ++j) {
            // reduce kap*(j+s0) mod n_os exactly before scaling to radians
            const long long t = ((long long)kap * (long long)(j + s0)) % n_os;
            const double ang = 2.0 * kPi * (double)t / n_os;
            M[(size_t)slot * L + j] = is_sin ? std::sin(ang) : std::cos(ang);
        }
    }
}

// Cyclic Jacobi rotations for a small symmetric matrix.
void sym_eig(int n, std::vector<double> &a, std::vector<double> &evals, std::vector<double> &evecs)
{
    std::vector<double> v((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double x = a[(size_t)i * n + j];
                tot += x * x;
                if (i != j) off += x * x;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return a[(size_t)x * n + x] < a[(size_t)y * n + y]; });
    evals.assign(n, 0.0);
    evecs.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        evals[j] = a[(size_t)order[j] * n + order[j]];
        for (int k = 0; k < n; ++k) evecs[(size_t)k * n + j] = v[(size_t)k * n + order[j]];
    }
}

}  // namespace ml
