// sem_model.cu -- the paper's performance model for splitting one homogeneous
// problem over several kinds of computing devices (section 4.1, Eq. 2-7).
//
// Execution time T = T_a + T_c; a device s_i computing cost C_i at its best
// performance P_opt(s_i) needs at least C_i / P_opt(s_i), so the run time of a
// split is bounded below by max_i C_i / P_opt(s_i).  The model's T_min is the
// minimum of that bound over the splits with sum_i C_i = C and C_i <= C_max(s_i)
// (device capacity, e.g. memory).  When the proportional split fits every
// capacity, T_min = C / sum_i P_opt(s_i) (performances add); otherwise some
// devices are filled to capacity and the rest share the remainder in
// proportion to their performance.  Host code only.
//
// Solution: f(T) = sum_i min(P_i T, Cmax_i) is continuous, piecewise linear and
// non-decreasing; T_min is the smallest T with f(T) >= C.  Devices saturate at
// t_i = Cmax_i / P_i; walking the t_i in increasing order, with S = the
// capacity of the saturated devices and Q = the performance of the others,
// T = (C - S) / Q is the answer as soon as it does not exceed the next t_i.

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "sem_common.cuh"

using namespace sem;

extern "C" {

int sem_perf_model(int ndev, const double *P_opt, const double *C_max, double C, double *T_min, double *C_split) {
    if (ndev < 1 || !P_opt || !T_min || !C_split) return fail(SEM_ERR_INVALID_ARG, "sem_perf_model: bad arguments");
    if (!(C >= 0.0) || !std::isfinite(C)) return fail(SEM_ERR_INVALID_ARG, "sem_perf_model: cost must be >= 0");
    std::vector<double> cap(ndev);
    for (int i = 0; i < ndev; ++i) {
        if (!(P_opt[i] > 0.0) || !std::isfinite(P_opt[i]))
            return fail(SEM_ERR_INVALID_ARG, "sem_perf_model: every P_opt must be > 0");
        cap[i] = (C_max && C_max[i] > 0.0) ? C_max[i] : INFINITY;
    }
    // devices in the order in which they saturate
    std::vector<int> ord(ndev);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return cap[a] / P_opt[a] < cap[b] / P_opt[b]; });
    double S = 0.0, Q = 0.0;
    for (int i = 0; i < ndev; ++i) Q += P_opt[i];
    double T = -1.0;
    int k = 0;  // devices ord[0..k) are saturated
    for (; k < ndev; ++k) {
        if (!(Q > 0.0)) break;  // only saturated devices left (rounding)
        const double t = (C - S) / Q;
        const int d = ord[k];
        if (t <= cap[d] / P_opt[d]) {
            T = t;
            break;
        }
        S += cap[d];
        Q -= P_opt[d];
    }
    if (T < 0.0) {
        // all devices full: feasible only if the capacities hold the cost exactly
        if (S < C) return fail(SEM_ERR_WORKSPACE, "sem_perf_model: the devices' capacities hold less than the cost");
        T = 0.0;
        for (int i = 0; i < ndev; ++i) T = std::max(T, cap[i] / P_opt[i]);
    }
    for (int i = 0; i < ndev; ++i) C_split[i] = std::min(P_opt[i] * T, cap[i]);
    *T_min = T;
    return SEM_OK;
}

}  // extern "C"
