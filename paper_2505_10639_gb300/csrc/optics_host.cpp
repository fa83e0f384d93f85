// Plan-time optics on the host. See optics_host.h.
#include "optics_host.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <stdexcept>

namespace mfbd_host {

namespace {

constexpr double kPi = 3.14159265358979323846;

// binomial coefficient, exact in 64-bit for the orders used here
uint64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

// R_n^m(rho) = sum_s (-1)^s (n-s)!/(s!((n+m)/2-s)!((n-m)/2-s)!) rho^(n-2s);
// the coefficient is the integer C(n-s, s) C(n-2s, (n-m)/2 - s).
double zernike_radial(int n, int m, double rho) {
    double acc = 0.0;
    for (int s = 0; s <= (n - m) / 2; ++s) {
        double c = (double)(binom(n - s, s) * binom(n - 2 * s, (n - m) / 2 - s));
        if (s & 1) c = -c;
        acc += c * std::pow(rho, (double)(n - 2 * s));
    }
    return acc;
}

// Kolmogorov phase spectrum constant A in W(f) = A r0^(-5/3) f^(-11/3),
// fixed by the structure function 2((24/5)Gamma(6/5))^(5/6) (r/r0)^(5/3).
double kolmogorov_psd_constant() {
    const double mu = 8.0 / 3.0;
    const double integral = -std::tgamma((1 - mu) / 2) / (std::pow(2.0, mu) * std::tgamma((1 + mu) / 2));
    const double dcoef = 2.0 * std::pow((24.0 / 5.0) * std::tgamma(6.0 / 5.0), 5.0 / 6.0);
    return dcoef / (4 * kPi * std::pow(2 * kPi, 5.0 / 3.0) * integral);
}

// Cyclic Jacobi eigen-decomposition of a symmetric matrix a[n][n] (row
// major). Returns eigenvalues in w and eigenvectors as the columns of v.
void jacobi_eigen(std::vector<double> a, int n, std::vector<double>& w, std::vector<double>& v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
                if (i == j) diag += x; else off += x;
            }
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // rotate columns p, q
                    double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rotate rows p, q
                    double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

// round to 10 significant digits (decimal), used to make the mode ordering
// insensitive to last-bit differences between eigen-solvers
double round_sig10(double x) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%.9e", x);
    return std::strtod(buf, nullptr);
}

}  // namespace

std::vector<uint8_t> pupil_mask(int n, float diam_px, float obscuration) {
    std::vector<uint8_t> m((size_t)n * n, 0);
    const double c = (n - 1) / 2.0;
    const double r = (double)diam_px * 0.5;
    const double ro = (double)obscuration * r;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double dx = x - c, dy = y - c;
            double r2 = dx * dx + dy * dy;
            bool in = r2 <= r * r;
            if (obscuration > 0.0f) in = in && r2 >= ro * ro;
            m[(size_t)y * n + x] = in ? 1 : 0;
        }
    return m;
}

void noll_to_nm(int j, int* n_out, int* m_out) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 < j) ++n;
    int p = j - n * (n + 1) / 2 - 1;
    int m = (n % 2 == 0) ? 2 * ((p + 1) / 2) : 2 * (p / 2) + 1;
    *n_out = n;
    *m_out = m;
}

double zernike(int j, double rho, double theta) {
    int n, m;
    noll_to_nm(j, &n, &m);
    double rad = zernike_radial(n, m, rho);
    if (m == 0) return std::sqrt((double)(n + 1)) * rad;
    double ang = (j % 2 == 0) ? std::cos(m * theta) : std::sin(m * theta);
    return std::sqrt(2.0 * (n + 1)) * rad * ang;
}

std::vector<double> noll_covariance(const std::vector<int>& js) {
    const size_t nj = js.size();
    std::vector<double> cov(nj * nj, 0.0);
    const double k = kolmogorov_psd_constant() * 8.0 * std::pow(kPi, 8.0 / 3.0) *
                     std::tgamma(14.0 / 3.0) / std::pow(2.0, 14.0 / 3.0);
    for (size_t u = 0; u < nj; ++u) {
        int n, m;
        noll_to_nm(js[u], &n, &m);
        for (size_t v = 0; v < nj; ++v) {
            int n2, m2;
            noll_to_nm(js[v], &n2, &m2);
            if (m != m2) continue;
            if (m != 0 && (js[u] % 2) != (js[v] % 2)) continue;
            double sign = (((n + n2 - 2 * m) / 2) % 2 == 0) ? 1.0 : -1.0;
            cov[u * nj + v] = k * sign * std::sqrt((double)(n + 1) * (n2 + 1)) *
                              std::tgamma((n + n2 - 5.0 / 3.0) / 2) /
                              (std::tgamma((n - n2 + 17.0 / 3.0) / 2) * std::tgamma((n2 - n + 17.0 / 3.0) / 2) *
                               std::tgamma((n + n2 + 23.0 / 3.0) / 2));
        }
    }
    return cov;
}

namespace {

void sample_modes(int n, float diam_px, const std::vector<uint8_t>& mask,
                  const std::vector<int>& js, std::vector<double>& zb) {
    const double c = (n - 1) / 2.0;
    const double r = (double)diam_px * 0.5;
    zb.assign(js.size() * (size_t)n * n, 0.0);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            if (!mask[(size_t)y * n + x]) continue;
            double rho = std::hypot(x - c, y - c) / r;
            double th = std::atan2(y - c, x - c);
            for (size_t i = 0; i < js.size(); ++i)
                zb[i * (size_t)n * n + (size_t)y * n + x] = zernike(js[i], rho, th);
        }
}

}  // namespace

ModalBasis zernike_basis(int n, float diam_px, float obscuration, int n_modes) {
    std::vector<uint8_t> mask = pupil_mask(n, diam_px, obscuration);
    std::vector<int> js;
    for (int j = 2; j < n_modes + 2; ++j) js.push_back(j);
    ModalBasis b;
    sample_modes(n, diam_px, mask, js, b.modes);
    std::vector<double> cov = noll_covariance(js);
    b.variance.resize(n_modes);
    for (int i = 0; i < n_modes; ++i) b.variance[i] = cov[(size_t)i * n_modes + i];
    return b;
}

ModalBasis kl_basis(int n, float diam_px, float obscuration, int n_modes) {
    int order = 0;
    while ((order + 1) * (order + 2) / 2 < 4 * n_modes + 1) ++order;
    const int jmax = (order + 1) * (order + 2) / 2;
    std::vector<int> js;
    for (int j = 2; j <= jmax; ++j) js.push_back(j);
    const size_t nj = js.size();
    std::vector<double> cov = noll_covariance(js);

    struct Entry { double ev, key; int m, kind; std::vector<double> vec; };
    std::vector<Entry> entries;
    // blocks by (m, kind): kind 0 = cos or m == 0, kind 1 = sin
    for (int m = 0; m <= order; ++m) {
        for (int kind = 0; kind < 2; ++kind) {
            if (m == 0 && kind == 1) continue;
            std::vector<int> idx;
            for (size_t i = 0; i < nj; ++i) {
                int nn, mm;
                noll_to_nm(js[i], &nn, &mm);
                int kk = (mm == 0 || js[i] % 2 == 0) ? 0 : 1;
                if (mm == m && kk == kind) idx.push_back((int)i);
            }
            if (idx.empty()) continue;
            const int nb = (int)idx.size();
            std::vector<double> sub((size_t)nb * nb);
            for (int a = 0; a < nb; ++a)
                for (int b = 0; b < nb; ++b) sub[(size_t)a * nb + b] = cov[(size_t)idx[a] * nj + idx[b]];
            std::vector<double> w, v;
            jacobi_eigen(sub, nb, w, v);
            for (int e = 0; e < nb; ++e) {
                std::vector<double> vec(nb);
                int big = 0;
                for (int a = 0; a < nb; ++a) {
                    vec[a] = v[(size_t)a * nb + e];
                    if (std::fabs(vec[a]) > std::fabs(vec[big])) big = a;
                }
                if (vec[big] < 0)
                    for (double& x : vec) x = -x;
                Entry en;
                en.ev = w[e];
                en.key = round_sig10(w[e]);
                en.m = m;
                en.kind = kind;
                en.vec.assign(nj, 0.0);
                for (int a = 0; a < nb; ++a) en.vec[idx[a]] = vec[a];
                entries.push_back(std::move(en));
            }
        }
    }
    std::stable_sort(entries.begin(), entries.end(), [](const Entry& a, const Entry& b) {
        if (a.key != b.key) return a.key > b.key;
        if (a.m != b.m) return a.m < b.m;
        return a.kind < b.kind;
    });
    if ((int)entries.size() < n_modes) throw std::runtime_error("too few KL modes");

    std::vector<uint8_t> mask = pupil_mask(n, diam_px, obscuration);
    std::vector<double> zb;
    sample_modes(n, diam_px, mask, js, zb);
    std::vector<size_t> pix;
    for (size_t i = 0; i < (size_t)n * n; ++i)
        if (mask[i]) pix.push_back(i);
    const size_t npup = pix.size();

    std::vector<std::vector<double>> q(n_modes, std::vector<double>(npup, 0.0));
    for (int i = 0; i < n_modes; ++i) {
        std::vector<double>& vi = q[i];
        for (size_t jz = 0; jz < nj; ++jz) {
            double cf = entries[i].vec[jz];
            if (cf == 0.0) continue;
            const double* z = &zb[jz * (size_t)n * n];
            for (size_t t = 0; t < npup; ++t) vi[t] += cf * z[pix[t]];
        }
        for (int p = 0; p < i; ++p) {  // modified Gram-Schmidt
            double dot = 0.0;
            for (size_t t = 0; t < npup; ++t) dot += q[p][t] * vi[t];
            dot /= (double)npup;
            for (size_t t = 0; t < npup; ++t) vi[t] -= dot * q[p][t];
        }
        double nrm = 0.0;
        for (size_t t = 0; t < npup; ++t) nrm += vi[t] * vi[t];
        nrm = std::sqrt(nrm / (double)npup);
        for (size_t t = 0; t < npup; ++t) vi[t] /= nrm;
    }
    ModalBasis b;
    b.modes.assign((size_t)n_modes * n * n, 0.0);
    b.variance.resize(n_modes);
    for (int i = 0; i < n_modes; ++i) {
        for (size_t t = 0; t < npup; ++t) b.modes[(size_t)i * n * n + pix[t]] = q[i][t];
        b.variance[i] = entries[i].ev;
    }
    return b;
}

std::vector<uint8_t> otf_support_half(const std::vector<uint8_t>& mask, int n) {
    std::vector<int> ys, xs;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            if (mask[(size_t)y * n + x]) { ys.push_back(y); xs.push_back(x); }
    std::vector<uint8_t> full((size_t)n * n, 0);
    for (size_t a = 0; a < ys.size(); ++a)
        for (size_t b = 0; b < ys.size(); ++b) {
            int dy = ((ys[a] - ys[b]) % n + n) % n;
            int dx = ((xs[a] - xs[b]) % n + n) % n;
            full[(size_t)dy * n + dx] = 1;
        }
    const int nh = n / 2 + 1;
    std::vector<uint8_t> half((size_t)n * nh);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < nh; ++x) half[(size_t)y * nh + x] = full[(size_t)y * n + x];
    return half;
}

}  // namespace mfbd_host
