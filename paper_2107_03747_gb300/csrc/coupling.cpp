// coupling.cpp -- host-side lattice normalisation N(c, Lt) (eq. latt_norm) and the coupling
// lambda_TGF (eq. lambdat_latt) from the measured E and Q of an ensemble.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/tgf.h"

namespace {
// N(c, Lt) depends only on (c, Lt, N): computed once per process (O(Lt^4) host work).
std::mutex g_norm_mu;
std::map<std::tuple<double, int, int>, double> g_norm_cache;
}  // namespace

static tgf_status norm_uncached(double c, int Lt, int N, double* norm_out);

extern "C" tgf_status tgf_norm(double c, int Lt, int N, double* norm_out) {
    if (!(c > 0) || !std::isfinite(c) || Lt < 2 || Lt > 512 || N < 2 || !norm_out) return TGF_EINVAL;
    const auto key = std::make_tuple(c, Lt, N);
    {
        std::lock_guard<std::mutex> lk(g_norm_mu);
        auto it = g_norm_cache.find(key);
        if (it != g_norm_cache.end()) {
            *norm_out = it->second;
            return TGF_OK;
        }
    }
    double v;
    tgf_status s = norm_uncached(c, Lt, N, &v);
    if (s != TGF_OK) return s;
    std::lock_guard<std::mutex> lk(g_norm_mu);
    g_norm_cache[key] = v;
    *norm_out = v;
    return TGF_OK;
}

static tgf_status norm_uncached(double c, int Lt, int N, double* norm_out) {
    const double pi = 3.14159265358979323846;
    // per-component tables: qhat_mu^2 = 4 sin^2(q/2), sin^2(q), cos^2(q/2) with q = 2 pi n / Lt
    std::vector<double> qh2(Lt), s2(Lt), c2(Lt);
    for (int n = 0; n < Lt; ++n) {
        const double q = 2.0 * pi * n / Lt;
        qh2[n] = 4.0 * std::sin(0.5 * q) * std::sin(0.5 * q);
        s2[n] = std::sin(q) * std::sin(q);
        c2[n] = std::cos(0.5 * q) * std::cos(0.5 * q);
    }
    const double a = 0.25 * c * c * (double)Lt * (double)Lt;
    double tot = 0.0;
    int nn[4];
    for (nn[0] = 0; nn[0] < Lt; ++nn[0])
        for (nn[1] = 0; nn[1] < Lt; ++nn[1]) {
            // primed sum: drop momenta whose two twisted-plane components are multiples of 2 pi N / Lt
            if (nn[0] % N == 0 && nn[1] % N == 0) continue;
            for (nn[2] = 0; nn[2] < Lt; ++nn[2]) {
                double part = 0.0;
                for (nn[3] = 0; nn[3] < Lt; ++nn[3]) {
                    const double qhat2 = qh2[nn[0]] + qh2[nn[1]] + qh2[nn[2]] + qh2[nn[3]];
                    double ang = 0.0;
                    for (int mu = 0; mu < 4; ++mu)
                        for (int nu = 0; nu < 4; ++nu)
                            if (mu != nu) ang += s2[nn[nu]] * c2[nn[mu]];
                    part += std::exp(-a * qhat2) / qhat2 * ang;
                }
                tot += part;
            }
        }
    const double inv = std::pow(c, 4) / 128.0 * tot;
    if (!(inv > 0)) return TGF_EINVAL;
    *norm_out = 1.0 / inv;
    return TGF_OK;
}

extern "C" tgf_status tgf_lambda(double c, int Lt, double t, const double* E, const double* Q, int ncfg,
                                 double* lambda_out, int* n_kept) {
    if (!E || !Q || ncfg < 1 || !lambda_out || !n_kept || !std::isfinite(t)) return TGF_EINVAL;
    double num = 0.0;
    int kept = 0;
    for (int i = 0; i < ncfg; ++i) {
        if (std::fabs(Q[i]) < 0.5) {  // delta_Q = 1 for |Q| < 1/2
            num += E[i];
            ++kept;
        }
    }
    *n_kept = kept;
    if (kept == 0) return TGF_ESTATE;
    double norm;
    tgf_status s = tgf_norm(c, Lt, 3, &norm);
    if (s != TGF_OK) return s;
    *lambda_out = norm * t * t * num / (3.0 * kept);
    return TGF_OK;
}

extern "C" tgf_status tgf_slice_correlator(const double* q, size_t q_stride, const double* Q, int ncfg, int T,
                                           double* C_out, int* n_kept) {
    if (!q || !Q || !C_out || !n_kept || ncfg < 1 || T < 1 || (size_t)T > q_stride) return TGF_EINVAL;
    // C(d) = <q(x0 + d) q(x0) delta_Q> / <delta_Q>, averaged over the source x0 (eq. qcorr)
    for (int d = 0; d < T; ++d) C_out[d] = 0.0;
    int kept = 0;
    for (int c = 0; c < ncfg; ++c) {
        if (!(std::fabs(Q[c]) < 0.5)) continue;
        ++kept;
        const double* qc = q + (size_t)c * q_stride;
        for (int d = 0; d < T; ++d) {
            double acc = 0.0;
            for (int x = 0; x < T; ++x) acc += qc[(x + d) % T] * qc[x];
            C_out[d] += acc / T;
        }
    }
    *n_kept = kept;
    if (kept == 0) return TGF_ESTATE;
    for (int d = 0; d < T; ++d) C_out[d] /= kept;
    return TGF_OK;
}
