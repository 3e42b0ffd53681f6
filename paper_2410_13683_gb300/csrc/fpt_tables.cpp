// fpt_tables.cpp -- host (FP64) model resolution and noise-table builder.
//
// Computes, for arXiv:2410.13683:
//   * the classical background, Eq. (2.21) without noise, in e-fold time:
//     phi' = pi, pi' = -(3 - pi^2/2)(pi + V'/V); H^2 = V/(3 - pi^2/2);
//   * the linear mode equation, Eq. (2.4), in e-fold time:
//     u'' + (3 - eps1) u' + [k^2/(aH)^2 + V''/H^2 - (3 - eps1) pi^2 - 2 pi pi'] u = 0,
//     from the Bunch-Davies state of Eq. (2.5) at N_sigma - ln(100/sigma);
//     the kink of Eq. (4.11) (V'' = V0 (a_+ - a_-) delta(phi - phi_*)) is
//     crossed with du/dN -> du/dN - (V0/H_T^2)(a_+ - a_-)/|pi_T| u;
//   * Bessel matching (Eq. 3.10) of the ansatz Eq. (3.5) at -k eta = sigma,
//     with d(-k eta)/dN = -(-k eta) and nu from the exact Eq. (3.13); the
//     growing mode of Eq. (3.11) gives the 1-D noise of Eq. (3.12):
//     S = (H/2pi)(2|B|/sqrt(pi)) Gamma(nu)/Gamma(3/2) (sigma/2)^(3/2-nu),
//     S_pi = (nu - 3/2) S;
//   * numerical matching (Eq. 3.9): the full covariance Xi of
//     (delta phi_k, delta pi_k) at k = sigma a H and its symmetric square root,
//     the noise matrix of the full-rank Langevin system, Eq. (2.24).
//
// Integrator: adaptive Dormand-Prince 5(4) (Dormand & Prince 1980); the
// background is stored at every accepted step and evaluated between steps by
// cubic Hermite interpolation. Bessel functions: std::cyl_bessel_j /
// std::cyl_neumann (C++17 special math).
#include "fpt_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <functional>
#include <limits>
#include <mutex>
#include <stdexcept>
#include <thread>
#include <vector>

namespace fpt_host {

static const double kPi = 3.14159265358979323846;
static const double kBdRatio = 100.0;  // k/(aH) at the Bunch-Davies start, times sigma

// ---------------------------------------------------------------------------
// Potential
// ---------------------------------------------------------------------------
// Gaussian bump, Eq. (4.12): V = V0 f (1 + g), f = phi^2/(m^2 + phi^2),
// g = K exp(-(phi - phi0)^2/(2 w^2)); f'/f = 2 m^2/(phi (m^2 + phi^2)),
// f''/f = 2 m^2 (m^2 - 3 phi^2)/(phi^2 (m^2 + phi^2)^2), g' = -g (phi - phi0)/w^2,
// g'' = g ((phi - phi0)^2/w^2 - 1)/w^2.
struct BumpTerms { double f1, f2, g, g1, g2, f; };

static BumpTerms bump_terms(const fpt_model &m, double phi)
{
    BumpTerms b;
    const double m2 = m.bump_m * m.bump_m, w2 = m.bump_width * m.bump_width, d = phi - m.bump_phi0;
    const double q = m2 + phi * phi;
    b.f = phi * phi / q;
    b.g = m.bump_K * std::exp(-0.5 * d * d / w2);
    b.f1 = 2.0 * m2 / (phi * q);
    b.f2 = 2.0 * m2 * (m2 - 3.0 * phi * phi) / (phi * phi * q * q);
    b.g1 = -b.g * d / w2;
    b.g2 = b.g * (d * d / w2 - 1.0) / w2;
    return b;
}

double dlnV(const fpt_model &m, double phi, int branch)
{
    if (m.kind == FPT_POT_EXP) return m.mu;
    if (m.kind == FPT_POT_BUMP) {
        const BumpTerms b = bump_terms(m, phi);
        return b.f1 + b.g1 / (1.0 + b.g);
    }
    bool above = branch == 0 ? (phi >= m.phi_star) : (branch > 0);
    double a = above ? m.a_plus : m.a_minus;
    return a / (1.0 + a * (phi - m.phi_star));
}

double Vof(const fpt_model &m, double phi, int branch)
{
    if (m.kind == FPT_POT_EXP) return m.V0 * std::exp(m.mu * phi);
    if (m.kind == FPT_POT_BUMP) {
        const BumpTerms b = bump_terms(m, phi);
        return m.V0 * b.f * (1.0 + b.g);
    }
    bool above = branch == 0 ? (phi >= m.phi_star) : (branch > 0);
    double a = above ? m.a_plus : m.a_minus;
    return m.V0 * (1.0 + a * (phi - m.phi_star));
}

// V''/V (away from the kink of the piecewise-linear potential, where it vanishes)
double d2V_over_V(const fpt_model &m, double phi)
{
    if (m.kind == FPT_POT_EXP) return m.mu * m.mu;
    if (m.kind == FPT_POT_BUMP) {
        const BumpTerms b = bump_terms(m, phi);
        return b.f2 + (2.0 * b.f1 * b.g1 + b.g2) / (1.0 + b.g);
    }
    return 0.0;
}

double hubble(const fpt_model &m, double phi, double pi, int branch)
{
    return std::sqrt(Vof(m, phi, branch) / (3.0 - 0.5 * pi * pi));
}

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4)
// ---------------------------------------------------------------------------
template <int D>
struct DP5 {
    using Vec = std::array<double, D>;
    using Rhs = std::function<void(double, const Vec &, Vec &)>;

    // One step of size h from (t, y) with f0 = f(t, y); returns y1, f1 and the
    // scaled error estimate.
    static double step(const Rhs &f, double t, const Vec &y, const Vec &f0, double h,
                       Vec &y1, Vec &f1, double rtol, const Vec &atol)
    {
        static const double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
        static const double a21 = 1.0 / 5;
        static const double a31 = 3.0 / 40, a32 = 9.0 / 40;
        static const double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
        static const double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187,
                            a53 = 64448.0 / 6561, a54 = -212.0 / 729;
        static const double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                            a64 = 49.0 / 176, a65 = -5103.0 / 18656;
        static const double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192,
                            b5 = -2187.0 / 6784, b6 = 11.0 / 84;
        // difference between the 5th- and 4th-order weights
        static const double e1 = 35.0 / 384 - 5179.0 / 57600, e3 = 500.0 / 1113 - 7571.0 / 16695,
                            e4 = 125.0 / 192 - 393.0 / 640, e5 = -2187.0 / 6784 + 92097.0 / 339200,
                            e6 = 11.0 / 84 - 187.0 / 2100, e7 = -1.0 / 40;
        Vec k2, k3, k4, k5, k6, tmp;
        for (int i = 0; i < D; ++i) tmp[i] = y[i] + h * a21 * f0[i];
        f(t + c2 * h, tmp, k2);
        for (int i = 0; i < D; ++i) tmp[i] = y[i] + h * (a31 * f0[i] + a32 * k2[i]);
        f(t + c3 * h, tmp, k3);
        for (int i = 0; i < D; ++i) tmp[i] = y[i] + h * (a41 * f0[i] + a42 * k2[i] + a43 * k3[i]);
        f(t + c4 * h, tmp, k4);
        for (int i = 0; i < D; ++i)
            tmp[i] = y[i] + h * (a51 * f0[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
        f(t + c5 * h, tmp, k5);
        for (int i = 0; i < D; ++i)
            tmp[i] = y[i] + h * (a61 * f0[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
        f(t + h, tmp, k6);
        for (int i = 0; i < D; ++i)
            y1[i] = y[i] + h * (b1 * f0[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
        f(t + h, y1, f1);
        double err = 0.0;
        for (int i = 0; i < D; ++i) {
            double e = h * (e1 * f0[i] + e3 * k3[i] + e4 * k4[i] + e5 * k5[i] + e6 * k6[i] + e7 * f1[i]);
            double sc = atol[i] + rtol * std::max(std::fabs(y[i]), std::fabs(y1[i]));
            err += (e / sc) * (e / sc);
        }
        return std::sqrt(err / D);
    }

    // Adaptive integration from t0 to t1 (t1 > t0). on_step(t, y, f) is
    // called for the initial point and every accepted step.
    // stop(t, y, f), when given, ends the integration after an accepted step.
    static void integrate(const Rhs &f, double t0, double t1, Vec &y, double rtol, const Vec &atol,
                          double h0, double hmax,
                          const std::function<void(double, const Vec &, const Vec &)> &on_step = nullptr,
                          const std::function<bool(double, const Vec &, const Vec &)> &stop = nullptr)
    {
        Vec f0, y1, f1;
        double t = t0, h = std::min(h0, t1 - t0);
        f(t, y, f0);
        if (on_step) on_step(t, y, f0);
        int guard = 0;
        while (t < t1) {
            if (++guard > 50000000) throw std::runtime_error("DP5: too many steps");
            bool last = false;
            if (t + h >= t1) { h = t1 - t; last = true; }
            double err = step(f, t, y, f0, h, y1, f1, rtol, atol);
            if (!(err <= 1.0)) {
                double fac = std::isfinite(err) ? std::max(0.2, 0.9 * std::pow(err, -0.2)) : 0.2;
                h *= fac;
                if (h < 1e-14 * std::max(1.0, std::fabs(t))) throw std::runtime_error("DP5: step underflow");
                continue;
            }
            t = last ? t1 : t + h;
            y = y1;
            f0 = f1;
            if (on_step) on_step(t, y, f0);
            if (stop && stop(t, y, f0)) return;
            double fac = err > 0 ? std::min(5.0, std::max(0.2, 0.9 * std::pow(err, -0.2))) : 5.0;
            h = std::min(h * fac, hmax);
        }
    }
};

// ---------------------------------------------------------------------------
// Background
// ---------------------------------------------------------------------------
struct BgPoint { double N, phi, pi, dphi, dpi; };

struct Background {
    std::vector<BgPoint> pre, post;  // pre: N < N_T (branch +), post: N >= N_T
    double N_T = std::numeric_limits<double>::quiet_NaN();
    bool kink = false;

    static void hermite(const BgPoint &a, const BgPoint &b, double N, double &phi, double &pi)
    {
        double h = b.N - a.N, s = (N - a.N) / h;
        double h00 = (1 + 2 * s) * (1 - s) * (1 - s), h10 = s * (1 - s) * (1 - s);
        double h01 = s * s * (3 - 2 * s), h11 = s * s * (s - 1);
        phi = h00 * a.phi + h10 * h * a.dphi + h01 * b.phi + h11 * h * b.dphi;
        pi = h00 * a.pi + h10 * h * a.dpi + h01 * b.pi + h11 * h * b.dpi;
    }

    static bool eval(const std::vector<BgPoint> &v, double N, double &phi, double &pi)
    {
        if (v.empty() || N < v.front().N || N > v.back().N) return false;
        auto it = std::upper_bound(v.begin(), v.end(), N,
                                   [](double x, const BgPoint &p) { return x < p.N; });
        size_t j = (it == v.begin()) ? 0 : size_t(it - v.begin()) - 1;
        if (j + 1 >= v.size()) j = v.size() - 2;
        hermite(v[j], v[j + 1], N, phi, pi);
        return true;
    }

    // Background state at N; branch = +1 before the kink, -1 after (0: none).
    void state(double N, double &phi, double &pi, int &branch) const
    {
        if (kink && N < N_T) {
            branch = +1;
            if (!eval(pre, N, phi, pi)) throw std::runtime_error("background: N out of range");
        } else {
            branch = kink ? -1 : 0;
            if (!eval(post, N, phi, pi)) throw std::runtime_error("background: N out of range");
        }
    }
    double N_max() const { return post.back().N; }
};

static const double kBgRtol = 1e-13;
static const double kBgHmax = 2e-3;

static void bg_rhs(const fpt_model &m, int branch, double, const std::array<double, 2> &y,
                   std::array<double, 2> &f)
{
    f[0] = y[1];
    f[1] = -(3.0 - 0.5 * y[1] * y[1]) * (y[1] + dlnV(m, y[0], branch));
}

static Background solve_background(const fpt_model &m, double phi0, double N_span)
{
    using D2 = DP5<2>;
    Background bg;
    std::array<double, 2> atol = {1e-16, 1e-18};
    std::array<double, 2> y = {phi0, -dlnV(m, phi0, 0)};
    bool has_kink = (m.kind == FPT_POT_PWLINEAR && phi0 > m.phi_star);
    auto push = [](std::vector<BgPoint> &v) {
        return [&v](double N, const std::array<double, 2> &yy, const std::array<double, 2> &ff) {
            v.push_back({N, yy[0], yy[1], ff[0], ff[1]});
        };
    };
    if (m.kind == FPT_POT_BUMP) {
        // smooth potential: N_T marks the onset of ultra-slow roll, the first
        // time eps2 = 2 pi'/pi reaches -3 (Sec. 4.3)
        D2::Rhs f = [&](double t, const std::array<double, 2> &yy, std::array<double, 2> &ff) {
            bg_rhs(m, 0, t, yy, ff);
        };
        // stop at the onset, or when inflation ends (eps1 = 1) without one
        auto usr = [](double, const std::array<double, 2> &yy, const std::array<double, 2> &ff) {
            return 2.0 * ff[1] / yy[1] <= -3.0 || 0.5 * yy[1] * yy[1] >= 1.0;
        };
        D2::integrate(f, 0.0, 400.0, y, kBgRtol, atol, 1e-4, kBgHmax, push(bg.post), usr);
        const size_t n = bg.post.size();
        if (n < 2 || !(2.0 * bg.post[n - 1].dpi / bg.post[n - 1].pi <= -3.0))
            throw std::runtime_error("the background never enters ultra-slow roll (eps2 > -3 throughout)");
        const BgPoint a = bg.post[n - 2], b = bg.post[n - 1];
        double lo = a.N, hi = b.N;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi), ph, pi;
            Background::hermite(a, b, mid, ph, pi);
            std::array<double, 2> ff;
            bg_rhs(m, 0, mid, {ph, pi}, ff);
            if (2.0 * ff[1] / pi > -3.0) lo = mid; else hi = mid;
        }
        bg.N_T = 0.5 * (lo + hi);
        bg.kink = false;
        // continue from the last accepted point (its duplicate is dropped)
        bg.post.pop_back();
        D2::integrate(f, b.N, bg.N_T + N_span, y, kBgRtol, atol, 1e-4, kBgHmax, push(bg.post));
        return bg;
    }
    if (!has_kink) {
        D2::Rhs f = [&](double t, const std::array<double, 2> &yy, std::array<double, 2> &ff) {
            bg_rhs(m, 0, t, yy, ff);
        };
        D2::integrate(f, 0.0, N_span, y, kBgRtol, atol, 1e-4, kBgHmax, push(bg.post));
        return bg;
    }
    bg.kink = true;
    D2::Rhs fp = [&](double t, const std::array<double, 2> &yy, std::array<double, 2> &ff) {
        bg_rhs(m, +1, t, yy, ff);
    };
    // Step until phi crosses phi_star, then land exactly on the crossing.
    std::array<double, 2> f0, y1, f1;
    double N = 0.0, h = 1e-4;
    fp(N, y, f0);
    bg.pre.push_back({N, y[0], y[1], f0[0], f0[1]});
    for (int guard = 0;; ++guard) {
        if (guard > 20000000 || N > N_span) throw std::runtime_error("background never reaches phi_star");
        double err = D2::step(fp, N, y, f0, h, y1, f1, kBgRtol, atol);
        if (!(err <= 1.0)) { h *= std::max(0.2, 0.9 * std::pow(err, -0.2)); continue; }
        if (y1[0] <= m.phi_star) {
            // root of the Hermite interpolant on this step, then an exact RK step
            BgPoint a = {N, y[0], y[1], f0[0], f0[1]}, b = {N + h, y1[0], y1[1], f1[0], f1[1]};
            double lo = a.N, hi = b.N;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), ph, pi;
                Background::hermite(a, b, mid, ph, pi);
                if (ph > m.phi_star) lo = mid; else hi = mid;
            }
            double hT = 0.5 * (lo + hi) - N;
            std::array<double, 2> yT, fT;
            if (hT > 0) D2::step(fp, N, y, f0, hT, yT, fT, kBgRtol, atol); else { yT = y; fT = f0; }
            bg.N_T = N + hT;
            bg.pre.push_back({bg.N_T, m.phi_star, yT[1], yT[1], fT[1]});
            y = {m.phi_star, yT[1]};
            break;
        }
        N += h;
        y = y1;
        f0 = f1;
        bg.pre.push_back({N, y[0], y[1], f0[0], f0[1]});
        h = std::min(h * std::min(5.0, std::max(0.2, 0.9 * std::pow(std::max(err, 1e-30), -0.2))), kBgHmax);
    }
    D2::Rhs fm = [&](double t, const std::array<double, 2> &yy, std::array<double, 2> &ff) {
        bg_rhs(m, -1, t, yy, ff);
    };
    D2::integrate(fm, bg.N_T, bg.N_T + N_span, y, kBgRtol, atol, 1e-4, kBgHmax, push(bg.post));
    return bg;
}

struct Resolved {
    fpt_model_info info;
    Background bg;
    double N_in = NAN, N_end = NAN;
    bool has_bg = false;
};

static Resolved resolve_full(const fpt_model &m)
{
    Resolved r;
    if (!std::isnan(m.n_in)) {
        const double span = m.kind == FPT_POT_BUMP ? m.n_end + 10.0 : std::max(60.0, 2.0 * m.n_end + 40.0);
        r.bg = solve_background(m, m.bg_phi0, span);
        r.has_bg = true;
        if (!r.bg.kink && m.kind != FPT_POT_BUMP) throw std::runtime_error("transition rule needs bg_phi0 > phi_star");
        r.N_in = r.bg.N_T + m.n_in;
        r.N_end = r.bg.N_T + m.n_end;
        int br;
        double ph, pi;
        r.bg.state(r.N_in, ph, pi, br);
        r.info.phi_in = ph;
        r.info.pi_in = pi;
        r.bg.state(r.N_end, ph, pi, br);
        r.info.phi_end = ph;
        r.info.N_T = r.bg.N_T;
    } else {
        r.info.phi_in = m.phi_in;
        r.info.pi_in = std::isnan(m.pi_in) ? -dlnV(m, m.phi_in, 0) : m.pi_in;
        r.info.phi_end = m.phi_end;
        r.info.N_T = NAN;
    }
    return r;
}

// Background time of the post-transition field value phi (monotone branch).
static double N_of_phi(const Background &bg, double phi, double N_lo, double N_hi)
{
    auto f = [&](double N) { double ph, pi; int br; bg.state(N, ph, pi, br); return ph - phi; };
    double flo = f(N_lo), fhi = f(N_hi);
    if (flo * fhi > 0) throw std::runtime_error("table phi outside the post-transition background");
    for (int it = 0; it < 200 && N_hi - N_lo > 1e-15 * std::max(1.0, std::fabs(N_lo)); ++it) {
        double mid = 0.5 * (N_lo + N_hi), fm = f(mid);
        if ((fm > 0) == (flo > 0)) { N_lo = mid; flo = fm; } else { N_hi = mid; }
    }
    return 0.5 * (N_lo + N_hi);
}

// ---------------------------------------------------------------------------
// Mode equation and Bessel matching
// ---------------------------------------------------------------------------
static void mode_rhs(const fpt_model &m, double k, int branch, double N,
                     const std::array<double, 6> &y, std::array<double, 6> &f)
{
    double phi = y[0], pi = y[1];
    double V = Vof(m, phi, branch);
    double H2 = V / (3.0 - 0.5 * pi * pi);
    double eps1 = 0.5 * pi * pi;
    double dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi, branch));
    double mass = (k * k) / (std::exp(2.0 * N) * H2) + d2V_over_V(m, phi) * V / H2
                  - (3.0 - eps1) * pi * pi - 2.0 * pi * dpi;
    f[0] = pi;
    f[1] = dpi;
    f[2] = y[3];
    f[3] = -(3.0 - eps1) * y[3] - mass * y[2];
    f[4] = y[5];
    f[5] = -(3.0 - eps1) * y[5] - mass * y[4];
}

static const double kModeRtol = 1e-11;

// Mode from its Bunch-Davies state at N0 to N1 (u(N0) = 1 normalisation).
static void evolve_mode(const fpt_model &m, const Background &bg, double k, double N0, double N1,
                        std::complex<double> &u, std::complex<double> &du)
{
    using D6 = DP5<6>;
    double ph0, pi0;
    int br0;
    bg.state(N0, ph0, pi0, br0);
    double kaH = k / (std::exp(N0) * hubble(m, ph0, pi0, br0));
    std::array<double, 6> y = {ph0, pi0, 1.0, -1.0, 0.0, -kaH};
    std::array<double, 6> atol = {1e-16, 1e-18, 1e-14, 1e-14, 1e-14, 1e-14};
    auto run = [&](double a, double b, int br) {
        D6::Rhs f = [&](double t, const std::array<double, 6> &yy, std::array<double, 6> &ff) {
            mode_rhs(m, k, br, t, yy, ff);
        };
        D6::integrate(f, a, b, y, kModeRtol, atol, 1e-4, 0.05);
    };
    if (bg.kink && N0 < bg.N_T && bg.N_T < N1) {
        run(N0, bg.N_T, +1);
        double piT = y[1];
        double HT2 = m.V0 / (3.0 - 0.5 * piT * piT);
        double jump = -(m.V0 / HT2) * (m.a_plus - m.a_minus) / std::fabs(piT);
        y[3] += jump * y[2];
        y[5] += jump * y[4];
        y[0] = m.phi_star;
        run(bg.N_T, N1, -1);
    } else {
        run(N0, N1, br0);
    }
    u = {y[2], y[4]};
    du = {y[3], y[5]};
}

static double nu_squared(const fpt_model &m, double phi, double pi, int branch)
{
    double eps1 = 0.5 * pi * pi;
    double dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi, branch));
    double eps2 = 2.0 * dpi / pi;
    double v1 = dlnV(m, phi, branch);
    return 2.25 - eps1 - 0.5 * eps1 * eps2 * eps2 / (3.0 - eps1) + (eps1 - 3.0) * (d2V_over_V(m, phi) - v1 * v1);
}

// Run fn(j) for j = 0 .. n-1 on a pool of host threads; the first exception
// stops the pool and is rethrown.
static void parallel_points(int n, const std::function<void(int)> &fn)
{
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::atomic<int> next(0);
    std::atomic<bool> failed(false);
    std::string err;
    std::mutex mu;
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) {
        pool.emplace_back([&]() {
            for (;;) {
                int j = next.fetch_add(1);
                if (j >= n || failed.load()) break;
                try {
                    fn(j);
                } catch (const std::exception &e) {
                    std::lock_guard<std::mutex> g(mu);
                    if (!failed.exchange(true)) err = e.what();
                }
            }
        });
    }
    for (auto &th : pool) th.join();
    if (failed) throw std::runtime_error(err);
}

// Bessel-matched noise (S, S_pi) of the mode that crosses sigma a H at
// background time Ns.
static void bessel_noise_at_N(const fpt_model &m, const Resolved &r, double Ns, double sigma,
                              double &S, double &Spi)
{
    const Background &bg = r.bg;
    if (!(Ns >= bg.N_T) || !(Ns <= bg.N_max())) throw std::runtime_error("table time outside the post-transition background");
    double ph, pi;
    int br;
    bg.state(Ns, ph, pi, br);
    double H = hubble(m, ph, pi, br);
    double k = sigma * std::exp(Ns) * H;
    double N0 = Ns - std::log(kBdRatio / sigma);
    if (N0 < 0.0) throw std::runtime_error("Bunch-Davies start precedes the background start");
    std::complex<double> u, du;
    evolve_mode(m, bg, k, N0, Ns, u, du);
    double nu = std::sqrt(nu_squared(m, ph, pi, br));
    // physical mode / p, with p = sqrt(-eta)/a = sqrt(z/k)/a and z = sigma
    double pref = std::exp(Ns - N0) / std::sqrt(2.0 * sigma);
    double z = sigma;
    double J = std::cyl_bessel_j(nu, z), Y = std::cyl_neumann(nu, z);
    // derivatives from the recurrence C'_nu = (nu/z) C_nu - C_{nu+1} (order >= 0)
    double Jp = (nu / z) * J - std::cyl_bessel_j(nu + 1.0, z);
    double Yp = (nu / z) * Y - std::cyl_neumann(nu + 1.0, z);
    std::complex<double> U = u * pref;                  // A J + B Y
    std::complex<double> Vv = -(1.5 * u + du) * pref / z;  // A J' + B Y'
    double W = J * Yp - Jp * Y;
    std::complex<double> B = (Vv * J - U * Jp) / W;
    S = (H / (2.0 * kPi)) * (2.0 * std::abs(B) / std::sqrt(kPi)) *
        (std::tgamma(nu) / std::tgamma(1.5)) * std::pow(0.5 * sigma, 1.5 - nu);
    Spi = (nu - 1.5) * S;
}

// Bessel-matched noise at field value phi (post-transition background).
static void bessel_noise(const fpt_model &m, const Resolved &r, double phi, double sigma,
                         double &S, double &Spi)
{
    bessel_noise_at_N(m, r, N_of_phi(r.bg, phi, r.bg.N_T, r.bg.N_max()), sigma, S, Spi);
}

// Full-rank noise of Eq. (3.9) at field value phi: Xi from the full mode
// (delta phi_k, delta pi_k = d delta phi_k / dN) of k = sigma a H at N_sigma,
// and S its symmetric square root: for a 2x2 positive semi-definite X with
// s = sqrt(det X), sqrt(X) = (X + s 1) / sqrt(tr X + 2 s).
static void numeric_noise(const fpt_model &m, const Resolved &r, double phi, double sigma,
                          double &Spp, double &Spq, double &Sqq)
{
    const Background &bg = r.bg;
    const double Ns = N_of_phi(bg, phi, bg.N_T, bg.N_max());
    double ph, pi;
    int br;
    bg.state(Ns, ph, pi, br);
    const double H = hubble(m, ph, pi, br);
    const double k = sigma * std::exp(Ns) * H;
    const double N0 = Ns - std::log(kBdRatio / sigma);
    if (N0 < 0.0) throw std::runtime_error("Bunch-Davies start precedes the background start");
    std::complex<double> u, du;
    evolve_mode(m, bg, k, N0, Ns, u, du);
    // physical mode = u / (exp(N0) sqrt(2k)); power k^3/(2 pi^2) |.|^2
    const double w = k * k * k / (2.0 * kPi * kPi) / (std::exp(2.0 * N0) * 2.0 * k);
    const double xpp = w * std::norm(u);
    const double xpq = w * (u.real() * du.real() + u.imag() * du.imag());
    const double xqq = w * std::norm(du);
    const double sd = std::sqrt(std::max(xpp * xqq - xpq * xpq, 0.0));
    const double den = std::sqrt(xpp + xqq + 2.0 * sd);
    if (!(den > 0.0)) { Spp = Spq = Sqq = 0.0; return; }
    Spp = (xpp + sd) / den;
    Spq = xpq / den;
    Sqq = (xqq + sd) / den;
}

// ---------------------------------------------------------------------------
// Entry points used by the C ABI
// ---------------------------------------------------------------------------
std::string validate_model(const fpt_model &m)
{
    if (m.kind != FPT_POT_PWLINEAR && m.kind != FPT_POT_EXP && m.kind != FPT_POT_BUMP) return "unknown potential kind";
    if (!(m.V0 > 0) || !std::isfinite(m.V0)) return "V0 must be positive and finite";
    if (!(m.dN > 0) || !std::isfinite(m.dN)) return "dN must be positive";
    if (m.max_steps < 1 || m.max_steps >= (int64_t(1) << 31)) return "max_steps out of [1, 2^31)";
    if (m.kind == FPT_POT_PWLINEAR) {
        if (!std::isfinite(m.a_plus) || !std::isfinite(m.a_minus) || !std::isfinite(m.phi_star))
            return "slopes and phi_star must be finite";
    } else if (m.kind == FPT_POT_EXP) {
        if (!std::isfinite(m.mu)) return "mu must be finite";
    } else {
        if (!std::isfinite(m.bump_K) || !(m.bump_K > -1.0) || !(m.bump_m > 0) || !std::isfinite(m.bump_m) ||
            !(m.bump_width > 0) || !std::isfinite(m.bump_width) || !std::isfinite(m.bump_phi0))
            return "bump parameters: need K > -1, m > 0, width > 0, finite phi0";
    }
    if (!std::isnan(m.n_in)) {
        if (m.kind == FPT_POT_EXP) return "the transition rule needs a piecewise-linear or bump potential";
        if (!(m.n_end > m.n_in) || !(m.n_in >= 0) || !(m.n_end < 200)) return "need 0 <= n_in < n_end < 200";
        if (m.kind == FPT_POT_PWLINEAR) {
            if (!(m.bg_phi0 > m.phi_star)) return "the transition rule needs bg_phi0 > phi_star";
            if (!(m.a_plus > 0) || !(m.a_minus > 0)) return "the transition rule needs positive slopes";
        } else if (!(m.bg_phi0 > 0) || !std::isfinite(m.bg_phi0)) {
            return "the transition rule needs a positive bg_phi0";
        }
    } else {
        if (!std::isfinite(m.phi_in) || !std::isfinite(m.phi_end)) return "phi_in and phi_end must be finite";
        if (!(m.phi_in > m.phi_end)) return "need phi_in > phi_end";
        if (m.kind == FPT_POT_BUMP && !(m.phi_end > 0)) return "the bump potential needs phi_end > 0";
        if (!std::isnan(m.pi_in) && !std::isfinite(m.pi_in)) return "pi_in must be finite or NaN";
    }
    return "";
}

fpt_model_info resolve(const fpt_model &m)
{
    return resolve_full(m).info;
}

void build_table(const fpt_model &m, int kind, int n_points, double sigma, double phi_lo,
                 double phi_hi, std::vector<double> &S, std::vector<double> &Spi,
                 double &lo_out, double &h_out)
{
    Resolved r = resolve_full(m);
    const bool by_time = kind == FPT_TABLE_BESSEL_N;
    if (by_time && (std::isnan(phi_lo) || std::isnan(phi_hi)))
        throw std::runtime_error("N-indexed tables need N_lo and N_hi");
    double lo = std::isnan(phi_lo) ? r.info.phi_end : phi_lo;
    double hi = std::isnan(phi_hi) ? r.info.phi_in : phi_hi;
    if (!(hi > lo)) throw std::runtime_error("need phi_hi > phi_lo");
    double h = (hi - lo) / (n_points - 1);
    lo_out = lo;
    h_out = h;
    S.assign(n_points, 0.0);
    Spi.assign(n_points, 0.0);
    if (kind == FPT_TABLE_DESITTER) {
        for (int j = 0; j < n_points; ++j) {
            double ph = lo + h * j;
            double pa = -dlnV(m, ph, 0);
            S[j] = std::sqrt(Vof(m, ph, 0) / (3.0 - 0.5 * pa * pa)) / (2.0 * kPi);
        }
        return;
    }
    if (kind != FPT_TABLE_BESSEL && kind != FPT_TABLE_BESSEL_N) throw std::runtime_error("unknown table kind");
    if (!r.has_bg) throw std::runtime_error("Bessel tables need the transition rule (n_in set)");
    if (!(sigma > 0 && sigma <= 10)) throw std::runtime_error("sigma out of (0, 10]");
    parallel_points(n_points, [&](int j) {
        if (by_time) bessel_noise_at_N(m, r, r.N_in + lo + h * j, sigma, S[j], Spi[j]);
        else bessel_noise(m, r, lo + h * j, sigma, S[j], Spi[j]);
    });
}

void build_table2(const fpt_model &m, int kind, int n_points, double sigma, double phi_lo,
                  double phi_hi, std::vector<double> &Spp, std::vector<double> &Spq,
                  std::vector<double> &Sqq, double &lo_out, double &h_out)
{
    if (kind != FPT_TABLE_NUMERIC) throw std::runtime_error("unknown 2-D table kind");
    Resolved r = resolve_full(m);
    if (!r.has_bg) throw std::runtime_error("numerical-matching tables need the transition rule (n_in set)");
    if (!(sigma > 0 && sigma <= 10)) throw std::runtime_error("sigma out of (0, 10]");
    double lo = std::isnan(phi_lo) ? r.info.phi_end : phi_lo;
    double hi = std::isnan(phi_hi) ? r.info.phi_in : phi_hi;
    if (!(hi > lo)) throw std::runtime_error("need phi_hi > phi_lo");
    double h = (hi - lo) / (n_points - 1);
    lo_out = lo;
    h_out = h;
    Spp.assign(n_points, 0.0);
    Spq.assign(n_points, 0.0);
    Sqq.assign(n_points, 0.0);
    parallel_points(n_points, [&](int j) { numeric_noise(m, r, lo + h * j, sigma, Spp[j], Spq[j], Sqq[j]); });
}

// ---------------------------------------------------------------------------
// Classical delta N (Sec. 2.2): linear power spectrum over the simulated mode
// range, its variance, and the constant-eps2 PDF
// ---------------------------------------------------------------------------
// P_R = k^3/(2 pi^2) |delta phi_k|^2 / (2 eps1), Eq. (2.8), of the mode with
// k = sigma a H at background time Ns, read at N_eval.
static double power_spectrum_at(const fpt_model &m, const Resolved &r, double Ns, double sigma,
                                double N_eval)
{
    const Background &bg = r.bg;
    double ph, pi;
    int br;
    bg.state(Ns, ph, pi, br);
    const double k = sigma * std::exp(Ns) * hubble(m, ph, pi, br);
    const double N0 = Ns - std::log(kBdRatio / sigma);
    if (N0 < 0.0) throw std::runtime_error("Bunch-Davies start precedes the background start");
    std::complex<double> u, du;
    evolve_mode(m, bg, k, N0, N_eval, u, du);
    double phe, pie;
    bg.state(N_eval, phe, pie, br);
    return k * k * k / (2.0 * kPi * kPi) * std::norm(u) / (std::exp(2.0 * N0) * 2.0 * k) / (pie * pie);
}

void power_spectrum(const fpt_model &m, double sigma, int n, const double *Ns, double N_eval, double *out)
{
    Resolved r = resolve_full(m);
    if (!r.has_bg) throw std::runtime_error("the power spectrum needs the transition rule (n_in set)");
    if (std::isnan(N_eval)) N_eval = r.N_end + 4.0;
    if (!(N_eval <= r.bg.N_max())) throw std::runtime_error("N_eval beyond the background");
    parallel_points(n, [&](int j) { out[j] = power_spectrum_at(m, r, Ns[j], sigma, N_eval); });
}

// sigma_R^2 = int P_R d ln k, Eq. (2.18), over the modes that reach sigma a H
// in [N_in, N_end]: d ln k = (1 - eps1) dN_s; composite Simpson rule on n_k
// (odd) points. Also eps2 = 2 pi'/pi of the background at N_in and N_end.
void classical_dn(const fpt_model &m, double sigma, int n_k, double N_eval, double &s2,
                  double &eps2_in, double &eps2_end, double &N_in, double &N_end)
{
    Resolved r = resolve_full(m);
    if (!r.has_bg) throw std::runtime_error("classical delta N needs the transition rule (n_in set)");
    if (std::isnan(N_eval)) N_eval = r.N_end + 4.0;
    if (!(N_eval <= r.bg.N_max())) throw std::runtime_error("N_eval beyond the background");
    std::vector<double> f(n_k);
    const double h = (r.N_end - r.N_in) / (n_k - 1);
    parallel_points(n_k, [&](int j) {
        const double N = r.N_in + h * j;
        double ph, pi;
        int br;
        r.bg.state(N, ph, pi, br);
        f[j] = power_spectrum_at(m, r, N, sigma, N_eval) * (1.0 - 0.5 * pi * pi);
    });
    double acc = f[0] + f[n_k - 1];
    for (int j = 1; j < n_k - 1; ++j) acc += (j & 1 ? 4.0 : 2.0) * f[j];
    s2 = acc * h / 3.0;
    auto eps2 = [&](double N) {
        double ph, pi;
        int br;
        r.bg.state(N, ph, pi, br);
        const double dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, ph, br));
        return 2.0 * dpi / pi;
    };
    eps2_in = eps2(r.N_in);
    eps2_end = eps2(r.N_end);
    N_in = r.N_in;
    N_end = r.N_end;
}

}  // namespace fpt_host
