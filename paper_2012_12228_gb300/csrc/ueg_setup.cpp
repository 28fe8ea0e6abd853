// Host-side setup of one UEG system: basis, momentum transfers, couplings,
// trial chemical potential (Sec. "Uniform Electron Gas", "Computational
// Details", and the FE trial of Sec. "Assessing the Phaseless Constraint").
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

#include "ftq_internal.h"

namespace ftq {
namespace {

using Vec3 = std::array<int, 3>;

int norm2(const Vec3& v) { return v[0] * v[0] + v[1] * v[1] + v[2] * v[2]; }

bool shell_order(const Vec3& a, const Vec3& b) {
    int na = norm2(a), nb = norm2(b);
    if (na != nb) return na < nb;
    return a < b;   // lexicographic (nx, ny, nz)
}

bool in_half_space(const Vec3& v) {
    for (int c : v)
        if (c != 0) return c > 0;
    return false;
}

// Occupation 1 / (1 + exp(beta (e - mu))), overflow-safe.
double fermi(double e, double mu, double beta) {
    double x = beta * (e - mu);
    if (x > 0) {
        double ex = std::exp(-x);
        return ex / (1.0 + ex);
    }
    return 1.0 / (1.0 + std::exp(x));
}

}  // namespace

std::string build_ueg(UegSetup& s, int N, int M, double rs, double theta, double mu, double dtau) {
    if (N <= 0 || M <= 0 || N >= 2 * M) return "need 0 < N < 2M";
    if (!(rs > 0) || !(theta > 0) || !(dtau > 0)) return "rs, theta and dtau must be positive";
    if (M > 4096) return "M too large (max 4096)";
    // closed shell: smallest ncut2 whose ball holds exactly M lattice points
    int ncut2 = -1;
    std::vector<Vec3> ball;
    for (int c2 = 0; c2 < 1024; ++c2) {
        int r = (int)std::floor(std::sqrt((double)c2) + 1e-9);
        ball.clear();
        for (int x = -r; x <= r; ++x)
            for (int y = -r; y <= r; ++y)
                for (int z = -r; z <= r; ++z) {
                    Vec3 v{x, y, z};
                    if (norm2(v) <= c2) ball.push_back(v);
                }
        if ((int)ball.size() == M) { ncut2 = c2; break; }
        if ((int)ball.size() > M) break;
    }
    if (ncut2 < 0) return "M is not a closed-shell plane-wave count";
    std::sort(ball.begin(), ball.end(), shell_order);

    s.N = N; s.M = M; s.ncut2 = ncut2;
    s.R = (int)std::floor(std::sqrt((double)ncut2) + 1e-9);
    s.rs = rs; s.theta = theta;
    const double pi = 3.14159265358979323846;
    s.L = std::cbrt(4.0 * pi * N / 3.0) * rs;
    s.Omega = s.L * s.L * s.L;
    s.TF = 0.5 * std::pow(9.0 * pi / 4.0, 2.0 / 3.0) / (rs * rs);
    s.beta = 1.0 / (theta * s.TF);
    s.n_slices = std::max(1, (int)std::lround(s.beta / dtau));
    s.dtau = s.beta / s.n_slices;
    const double kf = 2.0 * pi / s.L;

    s.nvec.resize(3 * M);
    s.eps.resize(M);
    for (int i = 0; i < M; ++i) {
        for (int d = 0; d < 3; ++d) s.nvec[3 * i + d] = ball[i][d];
        s.eps[i] = 0.5 * kf * kf * norm2(ball[i]);
    }

    // momentum transfers and their half space
    std::map<Vec3, int> half;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            Vec3 d{ball[i][0] - ball[j][0], ball[i][1] - ball[j][1], ball[i][2] - ball[j][2]};
            if (in_half_space(d)) half.emplace(d, 0);
        }
    std::vector<Vec3> hq;
    for (auto& kv : half) hq.push_back(kv.first);
    std::sort(hq.begin(), hq.end(), shell_order);
    for (size_t q = 0; q < hq.size(); ++q) half[hq[q]] = (int)q;
    s.nq_half = (int)hq.size();
    s.n_alpha = 2 * s.nq_half;
    s.qhalf.resize(3 * s.nq_half);
    s.cq.resize(s.nq_half);
    s.vq.resize(s.nq_half);
    for (int q = 0; q < s.nq_half; ++q) {
        for (int d = 0; d < 3; ++d) s.qhalf[3 * q + d] = hq[q][d];
        double q2 = kf * kf * norm2(hq[q]);
        s.vq[q] = 4.0 * pi / (s.Omega * q2);
        s.cq[q] = std::sqrt(2.0 * pi / (s.Omega * q2));
    }

    // slot map and pair lists
    const int nslot = 2 * s.nq_half + 1;
    s.vidx.assign((size_t)M * M, 0);
    std::vector<std::vector<std::pair<int, int>>> pairs(nslot);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            if (i == j) continue;
            Vec3 d{ball[i][0] - ball[j][0], ball[i][1] - ball[j][1], ball[i][2] - ball[j][2]};
            int slot;
            if (in_half_space(d)) {
                slot = 1 + 2 * half[d];
            } else {
                Vec3 m{-d[0], -d[1], -d[2]};
                slot = 2 + 2 * half[m];
            }
            s.vidx[(size_t)i * M + j] = (uint16_t)slot;
            pairs[slot].push_back({i, j});
        }
    if (nslot > 65535) return "too many momentum transfers for 16-bit slots";
    // difference cube: every n_i - n_k has components in [-2R, 2R]
    s.qS = 4 * s.R + 1;
    const int S = s.qS;
    s.qoff = 2 * s.R * (S * S + S + 1);
    s.pk.resize(M);
    for (int i = 0; i < M; ++i) s.pk[i] = ball[i][0] * S * S + ball[i][1] * S + ball[i][2];
    s.qcube.assign((size_t)S * S * S, 0);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) s.qcube[(size_t)(s.pk[i] - s.pk[j] + s.qoff)] = s.vidx[(size_t)i * M + j];
    s.pair_ptr.assign(nslot + 1, 0);
    s.pair_a.clear();
    s.pair_b.clear();
    for (int sl = 0; sl < nslot; ++sl) {
        s.pair_ptr[sl] = (int)s.pair_a.size();
        for (auto& p : pairs[sl]) {
            s.pair_a.push_back(p.first);
            s.pair_b.push_back(p.second);
        }
    }
    s.pair_ptr[nslot] = (int)s.pair_a.size();

    // one-body term left over by the sum of squares: 1/4 sum_Q (A^2 + B^2)
    // = V_ee + 1/(2 Omega) sum_Q v_Q sum_{K, K-Q in basis} n_K, so the
    // propagator's one-body part carries -1/(2 Omega) sum_{K' != K} 4 pi/|K-K'|^2.
    s.deps.assign(M, 0.0);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            if (i == j) continue;
            Vec3 d{ball[i][0] - ball[j][0], ball[i][1] - ball[j][1], ball[i][2] - ball[j][2]};
            s.deps[i] -= 0.5 * 4.0 * pi / (s.Omega * kf * kf * norm2(d));
        }

    // trial chemical potential: 2 sum_K f(eps_K; mu_T) = N by bisection
    double lo = *std::min_element(s.eps.begin(), s.eps.end()) - 50.0 / s.beta - 10.0;
    double hi = *std::max_element(s.eps.begin(), s.eps.end()) + 50.0 / s.beta + 10.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), n = 0;
        for (int i = 0; i < M; ++i) n += 2.0 * fermi(s.eps[i], mid, s.beta);
        if (n < N) lo = mid; else hi = mid;
    }
    s.mu_T = 0.5 * (lo + hi);
    s.mu = std::isnan(mu) ? s.mu_T : mu;
    // Madelung term: half of N * (-2.837297 / L), the value that reproduces
    // the printed N=2, M=7, r_s=3 FCI energy (Sec. Results).
    s.E_M = 0.5 * N * (-2.837297 / s.L);
    return "";
}

}  // namespace ftq
