// Host-side planning: w-bins by k-means (Section 3.1), supports from logical kernels
// (Section 3.2 footnote), memory and cost models (Eq. 9, Eq. 10) and the decision
// tree of Section 3.4 / Fig. 2.  Plain C++ on the host, FP64, multi-threaded.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>

#include "planner.h"

namespace rimo {
namespace planner {

static const int CANDIDATE_P[] = {1,  2,  3,  4,  5,  6,  8,  10,  12,  16,  20,
                                  24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256};

int hw_threads() {
    unsigned n = std::thread::hardware_concurrency();
    return n == 0 ? 1 : (int)std::min(n, 64u);
}

// Set in the worker threads of parallel_for: a parallel_for called from one of them runs
// serially, so nested loops never multiply the thread count.
static thread_local bool tl_worker = false;

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f, int64_t min_chunk) {
    int T = hw_threads();
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(T, n / std::max<int64_t>(1, min_chunk)));
    if (chunks <= 1 || tl_worker) {
        f(0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t step = (n + chunks - 1) / chunks;
    for (int64_t c = 0; c < chunks; ++c) {
        int64_t b = c * step, e = std::min(n, b + step);
        if (b < e)
            th.emplace_back([&f](int64_t lo, int64_t hi) {
                tl_worker = true;
                f(lo, hi);
            }, b, e);
    }
    for (auto& t : th) t.join();
}

std::vector<double> subset_w(const double* uvw, int64_t M, uint64_t seed, double fraction) {
    double frac = std::max(fraction, std::min(1.0, 4096.0 / (double)std::max<int64_t>(M, 1)));
    std::vector<double> out;
    if (frac >= 1.0) {
        out.resize(M);
        for (int64_t k = 0; k < M; ++k) out[k] = uvw[3 * k + 2];
        return out;
    }
    // the selection of each index is independent: chunks in parallel, joined in index order
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const int64_t chunk = 1 << 20, nch = (M + chunk - 1) / chunk;
    std::vector<std::vector<double>> part((size_t)nch);
    parallel_for(nch, [&](int64_t cb, int64_t ce) {
        for (int64_t c = cb; c < ce; ++c) {
            std::vector<double>& o = part[(size_t)c];
            o.reserve((size_t)(chunk * frac * 1.1) + 16);
            for (int64_t k = c * chunk; k < std::min(M, (c + 1) * chunk); ++k) {
                uint64_t st = seed + (uint64_t)(k + 1) * golden;
                double u = (double)(splitmix64(st) >> 11) * 0x1.0p-53;
                if (u < frac) o.push_back(uvw[3 * k + 2]);
            }
        }
    }, 1);
    size_t total = 0;
    for (const auto& o : part) total += o.size();
    out.reserve(total);
    for (const auto& o : part) out.insert(out.end(), o.begin(), o.end());
    return out;
}

// argmin_p |w - c_p| with ties to the lowest index (c ascending).
static inline int nearest_sorted(double w, const double* c, int P) {
    int lo = 0, hi = P;  // first index with c >= w
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (c[mid] < w) lo = mid + 1; else hi = mid;
    }
    int q = lo, best;
    if (q == 0) best = 0;
    else if (q == P) best = P - 1;
    else best = (std::fabs(w - c[q - 1]) <= std::fabs(w - c[q])) ? q - 1 : q;
    while (best > 0 && c[best - 1] == c[best]) --best;
    return best;
}

static inline int nearest_scan(double w, const double* c, int P) {
    int best = 0;
    double bd = std::fabs(w - c[0]);
    for (int p = 1; p < P; ++p) {
        double d = std::fabs(w - c[p]);
        if (d < bd) { bd = d; best = p; }
    }
    return best;
}

void nearest_all(const double* w, int64_t n, int64_t stride, const std::vector<double>& c,
                 int32_t* lab) {
    int P = (int)c.size();
    bool sorted = std::is_sorted(c.begin(), c.end());
    parallel_for(n, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) {
            double wk = w[k * stride];
            lab[k] = sorted ? nearest_sorted(wk, c.data(), P) : nearest_scan(wk, c.data(), P);
        }
    }, 1 << 14);
}

// Lloyd iterations with the labels assigned point by point (any centroid order).
static void lloyd_points(const std::vector<double>& w, std::vector<double>& c, int max_iter) {
    const int P = (int)c.size();
    const int64_t n = (int64_t)w.size();
    std::vector<int32_t> lab(n), nl(n);
    nearest_all(w.data(), n, 1, c, lab.data());
    std::vector<double> sum(P);
    std::vector<int64_t> cnt(P);
    for (int it = 0; it < max_iter; ++it) {
        std::fill(sum.begin(), sum.end(), 0.0);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t k = 0; k < n; ++k) { sum[lab[k]] += w[k]; cnt[lab[k]]++; }
        for (int p = 0; p < P; ++p)
            if (cnt[p]) c[p] = sum[p] / (double)cnt[p];
        nearest_all(w.data(), n, 1, c, nl.data());
        if (nl == lab) break;
        lab.swap(nl);
    }
}

// First index of each cluster's run in ascending data: with ascending centroids the nearest
// centroid (ties to the lower index) is non-decreasing in w, so cluster p holds exactly
// ws[b[p] .. b[p + 1]).  Returns false when the centroids are not ascending.
static bool cluster_runs(const std::vector<double>& ws, const std::vector<double>& c,
                         std::vector<int64_t>& b) {
    const int P = (int)c.size();
    const int64_t n = (int64_t)ws.size();
    if (!std::is_sorted(c.begin(), c.end())) return false;
    b[0] = 0;
    b[P] = n;
    for (int p = 1; p < P; ++p) {
        int64_t lo = b[p - 1], hi = n;
        while (lo < hi) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (nearest_sorted(ws[mid], c.data(), P) < p) lo = mid + 1; else hi = mid;
        }
        b[p] = lo;
    }
    return true;
}

std::vector<double> kmeans1d_sorted(const std::vector<double>& ws, int P, int max_iter) {
    const int64_t n = (int64_t)ws.size();
    std::vector<double> c(P);
    for (int p = 0; p < P; ++p) {
        int64_t idx = (int64_t)(((p + 0.5) * (double)n) / (double)P);
        c[p] = ws[std::min<int64_t>(n - 1, idx)];
    }
    // Each iteration takes the same labels as a point-by-point assignment, so the
    // iterations and the result are those of Lloyd's algorithm; a cluster's mean is summed
    // over its run in ascending order.  Centroids stay ascending (each mean lies inside its
    // own cell); should rounding ever break that, the point-by-point iterations take over.
    std::vector<int64_t> b(P + 1), nb(P + 1);
    if (!cluster_runs(ws, c, b)) {
        lloyd_points(ws, c, max_iter);
    } else {
        for (int it = 0; it < max_iter; ++it) {
            for (int p = 0; p < P; ++p) {
                if (b[p + 1] == b[p]) continue;  // an empty cluster keeps its centroid
                double s = 0.0;
                for (int64_t i = b[p]; i < b[p + 1]; ++i) s += ws[i];
                c[p] = s / (double)(b[p + 1] - b[p]);
            }
            if (!cluster_runs(ws, c, nb)) {
                lloyd_points(ws, c, max_iter - it - 1);
                break;
            }
            if (nb == b) break;
            b.swap(nb);
        }
    }
    std::sort(c.begin(), c.end());
    return c;
}

std::vector<double> kmeans1d(const std::vector<double>& w, int P, int max_iter) {
    std::vector<double> ws(w);
    std::sort(ws.begin(), ws.end());
    return kmeans1d_sorted(ws, P, max_iter);
}

// sqrt(1 - l^2 - m^2) - 1 in the cancellation-free form -s / (1 + sqrt(1 - s)).
double dn(double l, double m) {
    double s = l * l + m * m;
    return -s / (1.0 + std::sqrt(1.0 - s));
}

double wsclean_bound(const double* uvw, int64_t M, double fov_x, double fov_y) {
    const int64_t chunk = 1 << 20, nch = (M + chunk - 1) / chunk;
    std::vector<double> lo((size_t)nch), hi((size_t)nch);
    parallel_for(nch, [&](int64_t cb, int64_t ce) {
        for (int64_t c = cb; c < ce; ++c) {
            double l = uvw[3 * (c * chunk) + 2], h = l;
            for (int64_t k = c * chunk; k < std::min(M, (c + 1) * chunk); ++k) {
                double w = uvw[3 * k + 2];
                l = std::min(l, w);
                h = std::max(h, w);
            }
            lo[(size_t)c] = l;
            hi[(size_t)c] = h;
        }
    }, 1);
    double wl = *std::min_element(lo.begin(), lo.end()), wh = *std::max_element(hi.begin(), hi.end());
    return 2.0 * M_PI * (wh - wl) * (-dn(0.5 * fov_x, 0.5 * fov_y));
}

static double taper(double lam, double fov) {
    double a = std::fabs(lam), half = 0.5 * fov;
    if (a <= half) return 1.0;
    return 0.54 + 0.46 * std::cos(M_PI * (a - half) / half);
}

// Support of the residual kernel at offset w_r: smallest odd s <= max_wsupport whose
// centred s x s taps keep >= eta of the l2 norm of all L x L taps (norm by Parseval from
// the samples), or max_wsupport + 2 when even the cap keeps less (the cap truncates).
static int support_raw(double w_r, const KernelGeom& g) {
    int L = g.L, hm = g.max_wsupport / 2, ns = 2 * hm + 1;
    std::vector<std::complex<double>> c((size_t)L * L);
    double tot = 0.0;
    for (int a = 0; a < L; ++a) {
        double lam = (a - L / 2) * (2.0 * g.fov_x / L);
        double ta = taper(lam, g.fov_x);
        for (int b = 0; b < L; ++b) {
            double mu = (b - L / 2) * (2.0 * g.fov_y / L);
            double tb = taper(mu, g.fov_y);
            double ph = -2.0 * M_PI * w_r * dn(lam, mu);
            std::complex<double> ch(std::cos(ph), std::sin(ph));
            std::complex<double> v = g.literal ? (ta * tb) * ch : 1.0 + (ta * tb) * (ch - 1.0);
            c[(size_t)a * L + b] = v;
            tot += std::norm(v);
        }
    }
    tot /= (double)L * L;  // sum_t |K(t)|^2 = (1/L^2) sum |c|^2
    // central taps K(tx, ty), |t| <= hm: row pass over a, then column pass over b
    std::vector<std::complex<double>> E((size_t)L * ns), R((size_t)L * ns), K((size_t)ns * ns);
    for (int a = 0; a < L; ++a)
        for (int s = 0; s < ns; ++s) {
            double ang = 2.0 * M_PI * (double)(s - hm) * (double)(a - L / 2) / (double)L;
            E[(size_t)a * ns + s] = std::complex<double>(std::cos(ang), std::sin(ang));
        }
    for (int b = 0; b < L; ++b)
        for (int s = 0; s < ns; ++s) {
            std::complex<double> acc = 0.0;
            for (int a = 0; a < L; ++a) acc += c[(size_t)a * L + b] * E[(size_t)a * ns + s];
            R[(size_t)b * ns + s] = acc;
        }
    for (int sx = 0; sx < ns; ++sx)
        for (int sy = 0; sy < ns; ++sy) {
            std::complex<double> acc = 0.0;
            for (int b = 0; b < L; ++b) acc += R[(size_t)b * ns + sx] * E[(size_t)b * ns + sy];
            K[(size_t)sx * ns + sy] = acc / ((double)L * L);
        }
    double total = std::sqrt(tot);
    for (int s = 1; s <= g.max_wsupport; s += 2) {
        int h = s / 2;
        double e = 0.0;
        for (int x = hm - h; x <= hm + h; ++x)
            for (int y = hm - h; y <= hm + h; ++y) e += std::norm(K[(size_t)x * ns + y]);
        if (std::sqrt(e) >= g.eta * total) return s;
    }
    return g.max_wsupport + 2;
}

int support_at(double w_r, const KernelGeom& g) { return std::min(support_raw(w_r, g), g.max_wsupport); }

bool truncated_at(double w_r, const KernelGeom& g) {
    if (w_r == 0.0 || g.eta >= 1.0) return false;
    return support_raw(w_r, g) > g.max_wsupport;
}

std::vector<int32_t> support_table(double wr_max, const KernelGeom& g) {
    std::vector<int32_t> tab(N_SUPPORT_BINS, 1);
    if (wr_max <= 0.0) return tab;
    double step = wr_max / N_SUPPORT_BINS;
    std::vector<int32_t> raw(N_SUPPORT_BINS);
    parallel_for(N_SUPPORT_BINS, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) raw[q] = support_at((double)(q + 1) * step, g);
    }, 1);
    int run = 1;
    for (int q = 0; q < N_SUPPORT_BINS; ++q) { run = std::max(run, raw[q]); tab[q] = run; }
    return tab;
}

int support_bin(double abs_wr, double wr_max) {
    if (wr_max <= 0.0) return 0;
    double step = wr_max / N_SUPPORT_BINS;
    double q = std::floor(abs_wr / step);
    return q >= N_SUPPORT_BINS - 1 ? N_SUPPORT_BINS - 1 : (int)q;
}

// w_sub ascending (the subset's order does not change the model).
static ModelPoint model_for_P(const std::vector<double>& w_sub, int64_t M, int P,
                              const Params& pr) {
    std::vector<double> c = kmeans1d_sorted(w_sub, P, 100);
    int64_t n = (int64_t)w_sub.size();
    std::vector<int32_t> lab(n);
    nearest_all(w_sub.data(), n, 1, c, lab.data());
    std::vector<double> wr(n);
    double wr_max = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        wr[k] = w_sub[k] - c[lab[k]];
        wr_max = std::max(wr_max, std::fabs(wr[k]));
    }
    std::vector<int32_t> tab = support_table(wr_max, pr.kg);
    int64_t s2 = 0, s2p = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t S = tab[support_bin(std::fabs(wr[k]), wr_max)] + pr.J - 1;
        s2 += S * S;
        s2p += (S * S) + ((S * S) & 1);
    }
    double scale = (double)M / (double)n;
    ModelPoint mp;
    mp.P = P;
    mp.K = (double)s2 * scale;
    double KP = (double)s2p * scale;
    mp.m_G = 8.0 * KP + (double)META_BYTES_PER_VIS * (double)M;
    double Np = 4.0 * (double)pr.nx * (double)pr.ny;
    mp.cost = 2.0 * (10.0 * Np * std::log2(std::sqrt(Np)) * (double)P + 6.0 * mp.K);
    mp.truncated = truncated_at(wr_max, pr.kg);
    return mp;
}

Choice choose(const double* uvw, int64_t M, const Params& pr) {
    Choice ch;
    std::vector<double> w_sub = subset_w(uvw, M, pr.seed, pr.plan_fraction);
    ch.subset = (int64_t)w_sub.size();
    ch.wsclean = wsclean_bound(uvw, M, pr.kg.fov_x, pr.kg.fov_y);
    std::vector<int> cands;
    if (pr.n_wbins > 0) {
        cands.push_back(pr.n_wbins);
    } else {
        int pmax = std::max(1, (int)std::ceil(ch.wsclean));
        for (int p : CANDIDATE_P)
            if (p <= std::max(pmax, 1) && p <= std::max<int64_t>(1, ch.subset)) cands.push_back(p);
    }
    std::sort(w_sub.begin(), w_sub.end());
    ch.models.resize(cands.size());
    parallel_for((int64_t)cands.size(), [&](int64_t b, int64_t e) {  // independent models
        for (int64_t i = b; i < e; ++i) ch.models[(size_t)i] = model_for_P(w_sub, M, cands[(size_t)i], pr);
    }, 1);
    // With an automatic P only bin counts whose residual kernels fit the support cap keep
    // the eta norm fraction (Section 3.1); if none does, the largest candidate truncates
    // least.  A capped support makes K(P) flat in P, so cost alone would pick the fewest
    // bins however much of the kernels the cap cuts off.
    std::vector<const ModelPoint*> pool;
    for (const auto& m : ch.models)
        if (pr.n_wbins > 0 || !m.truncated) pool.push_back(&m);
    if (pool.empty()) {
        const ModelPoint* mx = &ch.models[0];
        for (const auto& m : ch.models)
            if (m.P > mx->P) mx = &m;
        pool.push_back(mx);
    }
    const ModelPoint* best = pool[0];
    for (const ModelPoint* m : pool)
        if (m->cost < best->cost || (m->cost == best->cost && m->P < best->P)) best = m;
    ch.p_star = best->P;
    ch.est_m_g = best->m_G;
    ch.est_cost = best->cost;
    double budget = (double)pr.budget;
    if (pr.mode != RIMO_MODE_AUTO) {
        ch.P = best->P;
        ch.mode = pr.mode;
        return ch;
    }
    if (pr.budget <= 0 || best->m_G <= budget) {
        ch.P = best->P;
        ch.mode = RIMO_MODE_STORED_G;
        return ch;
    }
    // under the budget: the nearest P to P* that fits, kernels within the cap preferred
    const ModelPoint* pick = nullptr;
    std::vector<const ModelPoint*> all;
    for (const auto& m : ch.models) all.push_back(&m);
    for (const auto* set : {&pool, &all}) {
        for (const ModelPoint* m : *set) {
            if (m->m_G > budget) continue;
            if (!pick) { pick = m; continue; }
            int d = std::abs(m->P - best->P), dp = std::abs(pick->P - best->P);
            if (d < dp || (d == dp && m->P < pick->P)) pick = m;
        }
        if (pick) break;
    }
    if (pick) {
        ch.P = pick->P;
        ch.mode = RIMO_MODE_STORED_G;
        ch.est_m_g = pick->m_G;
        ch.est_cost = pick->cost;
        return ch;
    }
    double mmin = ch.models[0].m_G;
    for (const auto& m : ch.models) mmin = std::min(mmin, m.m_G);
    const ModelPoint* st = nullptr;
    for (const auto& m : ch.models)
        if (m.m_G <= 1.05 * mmin && (!st || m.P < st->P)) st = &m;
    ch.P = st->P;
    ch.mode = RIMO_MODE_HOLOGRAPHIC;
    ch.check_h = true;
    ch.est_m_g = st->m_G;
    ch.est_cost = st->cost;
    return ch;
}

}  // namespace planner
}  // namespace rimo
