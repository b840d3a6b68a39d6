// Host-side FP64 linear algebra for the index build: the symmetric eigendecomposition of
// Alg. 1 step 4 and the eigensystem allocation of Alg. 2. Also error reporting helpers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "taco_internal.h"

namespace taco {

static thread_local std::string g_last_error;
thread_local const char* g_launch_step = "";

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    int code = (e == cudaErrorMemoryAllocation) ? TACO_ENOMEM : TACO_ECUDA;
    const char* step = g_launch_step;
    g_launch_step = "";
    return fail(code, "%s failed%s%s: %s (%s:%d)", what, *step ? " at " : "", step, cudaGetErrorString(e),
                file, line);
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Cyclic Jacobi eigenvalue method for a symmetric matrix (Golub & Van Loan, "Matrix
// Computations", Sec. 8.5: the symmetric Schur decomposition by plane rotations).
// a: [d][d] row-major, destroyed. vecs: [d][d], column j is the eigenvector of vals[j].
void jacobi_eigen(int d, std::vector<double>& a, std::vector<double>& vecs,
                  std::vector<double>& vals) {
    vecs.assign(size_t(d) * d, 0.0);
    for (int i = 0; i < d; ++i) vecs[size_t(i) * d + i] = 1.0;
    double frob = 0.0;
    for (double v : a) frob += v * v;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) off += a[size_t(p) * d + q] * a[size_t(p) * d + q];
        if (off <= 1e-30 * frob || off == 0.0) break;
        for (int p = 0; p < d - 1; ++p) {
            for (int q = p + 1; q < d; ++q) {
                const double apq = a[size_t(p) * d + q];
                if (apq == 0.0) continue;
                const double app = a[size_t(p) * d + p];
                const double aqq = a[size_t(q) * d + q];
                const double tau = (aqq - app) / (2.0 * apq);
                double t;
                if (std::fabs(tau) > 1e150) {
                    t = 0.5 / tau;
                } else {
                    t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                }
                const double c = 1.0 / std::sqrt(1.0 + t * t);
                const double s = t * c;
                // A <- A J : columns p and q
                for (int k = 0; k < d; ++k) {
                    const double akp = a[size_t(k) * d + p], akq = a[size_t(k) * d + q];
                    a[size_t(k) * d + p] = c * akp - s * akq;
                    a[size_t(k) * d + q] = s * akp + c * akq;
                }
                // A <- J^T A : rows p and q
                for (int k = 0; k < d; ++k) {
                    const double apk = a[size_t(p) * d + k], aqk = a[size_t(q) * d + k];
                    a[size_t(p) * d + k] = c * apk - s * aqk;
                    a[size_t(q) * d + k] = s * apk + c * aqk;
                }
                a[size_t(p) * d + q] = 0.0;
                a[size_t(q) * d + p] = 0.0;
                // V <- V J
                for (int k = 0; k < d; ++k) {
                    const double vkp = vecs[size_t(k) * d + p], vkq = vecs[size_t(k) * d + q];
                    vecs[size_t(k) * d + p] = c * vkp - s * vkq;
                    vecs[size_t(k) * d + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    vals.resize(d);
    for (int i = 0; i < d; ++i) vals[i] = a[size_t(i) * d + i];
}

// Alg. 2 (Eigensystem Allocation). lam: eigenvalues, any order. Buckets receive indices
// into lam. Eigenvalues are scaled by 1/lambda_min (floored at 1e-12 lambda_max) so that
// all are >= 1 (step 3), ordered descending with ties kept in index order (step 4), and
// each of the N_s*s largest goes to the non-full bucket with the smallest product
// (steps 5-8; products tracked as sums of logarithms, ties to the lowest bucket index).
void eigensystem_allocation(const std::vector<double>& lam, int n_subspaces, int sub_dim,
                            std::vector<std::vector<int>>& buckets) {
    const int d = int(lam.size());
    double mx = lam[0], mn = lam[0];
    for (double v : lam) {
        mx = std::max(mx, v);
        mn = std::min(mn, v);
    }
    const double floor_v = std::max(mn, 1e-12 * mx);
    std::vector<double> scaled(d);
    for (int i = 0; i < d; ++i) scaled[i] = std::max(lam[i], floor_v) / floor_v;
    std::vector<int> order(d);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return scaled[x] > scaled[y]; });
    buckets.assign(n_subspaces, {});
    std::vector<double> logp(n_subspaces, 0.0);
    for (int i = 0; i < n_subspaces * sub_dim; ++i) {
        int best = -1;
        for (int j = 0; j < n_subspaces; ++j) {
            if (int(buckets[j].size()) < sub_dim && (best < 0 || logp[j] < logp[best])) best = j;
        }
        buckets[best].push_back(order[i]);
        logp[best] += std::log(scaled[order[i]]);
    }
}

}  // namespace taco

extern "C" const char* taco_last_error(void) { return taco::g_last_error.c_str(); }
