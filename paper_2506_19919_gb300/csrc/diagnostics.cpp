// Host-side convergence diagnostics of HMC output (Sec. 4 checks R-hat < 1.2):
// multi-chain effective sample size with Geyer's initial monotone sequence and
// split R-hat (Gelman et al., Bayesian Data Analysis, 3rd ed., Sec. 11.4-11.5).
// FP64; galaxies are spread over host threads.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "../../include/sps.h"

namespace {

// draws x[m * n + t] of M chains, N draws each.
double ess_one(const double* x, int M, int N) {
    if (N < 4) return (double)M * N;
    std::vector<double> mean(M, 0.0), var(M, 0.0);
    for (int m = 0; m < M; ++m) {
        double s = 0.0;
        for (int t = 0; t < N; ++t) s += x[(size_t)m * N + t];
        mean[m] = s / N;
        double v = 0.0;
        for (int t = 0; t < N; ++t) {
            double d = x[(size_t)m * N + t] - mean[m];
            v += d * d;
        }
        var[m] = v / (N - 1.0);
    }
    double W = 0.0, gm = 0.0;
    for (int m = 0; m < M; ++m) {
        W += var[m];
        gm += mean[m];
    }
    W /= M;
    gm /= M;
    double var_plus = W * (N - 1.0) / N;
    if (M > 1) {
        double b = 0.0;
        for (int m = 0; m < M; ++m) b += (mean[m] - gm) * (mean[m] - gm);
        var_plus += b / (M - 1.0);
    }
    if (!(var_plus > 0.0) || !std::isfinite(var_plus)) return (double)M * N;
    // autocovariance (biased, per chain) at lag t, averaged over chains
    auto acov = [&](int lag) {
        double s = 0.0;
        for (int m = 0; m < M; ++m) {
            const double* c = x + (size_t)m * N;
            double a = 0.0;
            for (int t = 0; t + lag < N; ++t) a += (c[t] - mean[m]) * (c[t + lag] - mean[m]);
            s += a / N;
        }
        return s / M;
    };
    auto rho = [&](int lag) { return lag == 0 ? 1.0 : 1.0 - (W - acov(lag)) / var_plus; };
    double tau = -1.0, prev = INFINITY;
    for (int k = 0; k + 1 < N; k += 2) {
        double pk = rho(k) + rho(k + 1);
        if (pk < 0.0) break;
        pk = std::min(pk, prev);
        prev = pk;
        tau += 2.0 * pk;
    }
    tau = std::max(tau, 1.0 / std::log10((double)M * N));
    return (double)M * N / tau;
}

double rhat_one(const double* x, int M, int N) {
    const int h = N / 2;
    if (h < 2) return NAN;
    const int MM = 2 * M;
    std::vector<double> mean(MM), var(MM);
    for (int m = 0; m < M; ++m)
        for (int part = 0; part < 2; ++part) {
            const double* c = x + (size_t)m * N + (part ? N - h : 0);
            double s = 0.0;
            for (int t = 0; t < h; ++t) s += c[t];
            double mu = s / h, v = 0.0;
            for (int t = 0; t < h; ++t) v += (c[t] - mu) * (c[t] - mu);
            mean[2 * m + part] = mu;
            var[2 * m + part] = v / (h - 1.0);
        }
    double W = 0.0, gm = 0.0;
    for (int i = 0; i < MM; ++i) {
        W += var[i];
        gm += mean[i];
    }
    W /= MM;
    gm /= MM;
    double b = 0.0;
    for (int i = 0; i < MM; ++i) b += (mean[i] - gm) * (mean[i] - gm);
    const double B = h * b / (MM - 1.0);
    const double vp = (h - 1.0) / h * W + B / h;
    return W > 0.0 ? std::sqrt(vp / W) : INFINITY;
}

}  // namespace

extern "C" sps_status sps_diagnostics(const float* samples, int64_t n_gal, int32_t chains_per_gal,
                                      int32_t n_draws, int32_t n_param, double* ess_out,
                                      double* rhat_out) {
    if (!samples || n_gal <= 0 || chains_per_gal < 1 || n_draws < 1 || n_param < 1)
        return SPS_E_INVALID_ARG;
    const int M = chains_per_gal, N = n_draws, P = n_param;
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    nt = (unsigned)std::min<int64_t>(nt, n_gal);
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nt; ++w) {
        pool.emplace_back([=]() {
            std::vector<double> buf((size_t)M * N);
            for (int64_t g = w; g < n_gal; g += nt) {
                for (int p = 0; p < P; ++p) {
                    for (int m = 0; m < M; ++m)
                        for (int t = 0; t < N; ++t)
                            buf[(size_t)m * N + t] =
                                samples[(((size_t)g * M + m) * N + t) * P + p];
                    if (ess_out) ess_out[g * P + p] = ess_one(buf.data(), M, N);
                    if (rhat_out) rhat_out[g * P + p] = rhat_one(buf.data(), M, N);
                }
            }
        });
    }
    for (auto& t : pool) t.join();
    return SPS_OK;
}
