// Host-side planning declarations (Section 3.1, Section 3.4).
#pragma once

#include <stdint.h>

#include <functional>
#include <vector>

#include "rimo.h"

namespace rimo {
namespace planner {

constexpr int N_SUPPORT_BINS = 64;

// SplitMix64 output function (Steele, Lea & Flood 2014).
inline uint64_t splitmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
constexpr int META_BYTES_PER_VIS = 16;

struct KernelGeom {
    int L = 64;
    int max_wsupport = 9;
    double fov_x = 0, fov_y = 0;
    double eta = 0.9999;
    bool literal = false;
};

struct Params {
    int nx = 0, ny = 0, J = 7;
    KernelGeom kg;
    uint64_t seed = 0;
    double plan_fraction = 0.01;
    int n_wbins = 0;
    int mode = 0;
    int64_t budget = 0;
};

struct ModelPoint {
    int P = 0;
    double K = 0, m_G = 0, cost = 0;
    bool truncated = false;  // the support cap cuts the kernel at the largest residual w
};

struct Choice {
    int P = 1;
    int mode = RIMO_MODE_STORED_G;
    int p_star = 1;
    bool check_h = false;
    int64_t subset = 0;
    double wsclean = 0, est_m_g = 0, est_cost = 0;
    std::vector<ModelPoint> models;
};

int hw_threads();
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f, int64_t min_chunk);
std::vector<double> subset_w(const double* uvw, int64_t M, uint64_t seed, double fraction);
void nearest_all(const double* w, int64_t n, int64_t stride, const std::vector<double>& c,
                 int32_t* lab);
std::vector<double> kmeans1d(const std::vector<double>& w, int P, int max_iter);
std::vector<double> kmeans1d_sorted(const std::vector<double>& ws, int P, int max_iter);
double dn(double l, double m);
double wsclean_bound(const double* uvw, int64_t M, double fov_x, double fov_y);
int support_at(double w_r, const KernelGeom& g);
bool truncated_at(double w_r, const KernelGeom& g);
std::vector<int32_t> support_table(double wr_max, const KernelGeom& g);
int support_bin(double abs_wr, double wr_max);
Choice choose(const double* uvw, int64_t M, const Params& pr);

}  // namespace planner
}  // namespace rimo
