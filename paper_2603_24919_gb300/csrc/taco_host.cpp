// Host-side FP64 linear algebra for the index build: the symmetric eigendecomposition of
// Alg. 1 step 4 and the eigensystem allocation of Alg. 2. Also error reporting helpers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
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

// Symmetric eigendecomposition A = V diag(vals) V^T in two stages (Golub & Van Loan, "Matrix
// Computations", Sec. 8.3): (1) Householder reduction to tridiagonal form, A = Q T Q^T, with
// Q accumulated; (2) implicit symmetric QR steps with the Wilkinson shift on T, deflating
// off-diagonal entries below eps (|t_ii| + |t_i+1,i+1|), each step's Givens rotations applied
// to Q. O(d^3) with a small constant: a 960 x 960 covariance takes about a second.
// a: [d][d] row-major symmetric, destroyed. vecs: [d][d], column j is the eigenvector of
// vals[j] (vals in no particular order).
void symmetric_eigen(int d, std::vector<double>& a, std::vector<double>& vecs, std::vector<double>& vals) {
    auto A = [&](int i, int j) -> double& { return a[size_t(i) * d + j]; };
    vals.assign(d, 0.0);
    vecs.assign(size_t(d) * d, 0.0);
    if (d == 0) return;
    std::vector<double> diag(d), off(d, 0.0);   // T: diag[i], off[i] = T(i+1, i)
    // (1) Householder: for column k, a reflector P = I - beta v v^T on rows/cols k+1 .. d-1
    // zeroes A(k+2 .., k). The reflectors are kept (v in the column below the subdiagonal,
    // beta separately) and applied to the identity afterwards, last first.
    std::vector<double> betas(d, 0.0), v(d), p(d), w(d);
    for (int k = 0; k + 2 < d; ++k) {
        const int m = d - k - 1;   // length of x = A(k+1 .., k)
        double sigma = 0.0;
        for (int i = 1; i < m; ++i) sigma += A(k + 1 + i, k) * A(k + 1 + i, k);
        const double x0 = A(k + 1, k);
        if (sigma == 0.0) {   // already zero below the subdiagonal
            betas[k] = 0.0;
            continue;
        }
        const double mu = std::sqrt(x0 * x0 + sigma);
        // v = x - mu e1 (P x = mu e1), its first entry computed without cancellation, then
        // scaled so that v0 = 1
        const double v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
        const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = A(k + 1 + i, k) / v0;
        // p = beta A22 v, w = p - (beta p^T v / 2) v, A22 -= v w^T + w v^T
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            const double* row = &A(k + 1 + i, k + 1);
            for (int j = 0; j < m; ++j) t += row[j] * v[j];
            p[i] = beta * t;
        }
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += p[i] * v[i];
        const double c = 0.5 * beta * pv;
        for (int i = 0; i < m; ++i) w[i] = p[i] - c * v[i];
        for (int i = 0; i < m; ++i) {
            double* row = &A(k + 1 + i, k + 1);
            const double vi = v[i], wi = w[i];
            for (int j = 0; j < m; ++j) row[j] -= vi * w[j] + wi * v[j];
        }
        A(k + 1, k) = mu;   // P x = mu e1
        A(k, k + 1) = mu;
        for (int i = 1; i < m; ++i) A(k + 1 + i, k) = v[i];   // keep v (v0 = 1 implied)
        for (int i = 1; i < m; ++i) A(k, k + 1 + i) = 0.0;
        betas[k] = beta;
    }
    for (int i = 0; i < d; ++i) diag[i] = A(i, i);
    for (int i = 0; i + 1 < d; ++i) off[i] = A(i + 1, i);
        // Q = P_0 P_1 ... P_{d-3}: start from I and apply P_k from the left, last k first. Q is
    // kept transposed (Qt[j][i] = Q(i, j)) so that both stages update contiguous rows.
    std::vector<double> Qt(size_t(d) * d, 0.0);
    for (int i = 0; i < d; ++i) Qt[size_t(i) * d + i] = 1.0;
    for (int k = d - 3; k >= 0; --k) {
        const double beta = betas[k];
        if (beta == 0.0) continue;
        const int m = d - k - 1;
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = A(k + 1 + i, k);
        // rows k+1 .. of Q: Q -= beta v (v^T Q), columns k+1 .. only (the rest is still I)
        for (int j = k + 1; j < d; ++j) {
            double* qj = &Qt[size_t(j) * d + k + 1];
            double t = 0.0;
            for (int i = 0; i < m; ++i) t += v[i] * qj[i];
            t *= beta;
            if (t == 0.0) continue;
            for (int i = 0; i < m; ++i) qj[i] -= t * v[i];
        }
    }
    // (2) implicit symmetric QR with the Wilkinson shift on the unreduced blocks of T
    const double eps = std::numeric_limits<double>::epsilon();
    int hi = d - 1;
    int iters = 0;
    const int max_iters = 60 * d;
    std::vector<double> tmp(d);
    while (hi > 0) {
        // deflate negligible off-diagonal entries from the bottom
        for (int i = 0; i < hi; ++i)
            if (std::fabs(off[i]) <= eps * (std::fabs(diag[i]) + std::fabs(diag[i + 1]))) off[i] = 0.0;
        while (hi > 0 && off[hi - 1] == 0.0) --hi;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && off[lo - 1] != 0.0) --lo;   // T(lo .. hi) is unreduced
        if (++iters > max_iters) break;              // (not reached for a symmetric input)
        // Wilkinson shift from the trailing 2 x 2 block
        const double dd = 0.5 * (diag[hi - 1] - diag[hi]);
        const double e2 = off[hi - 1] * off[hi - 1];
        const double denom = dd + (dd >= 0.0 ? 1.0 : -1.0) * std::sqrt(dd * dd + e2);
        const double mu = denom != 0.0 ? diag[hi] - e2 / denom : diag[hi];
        double x = diag[lo] - mu, z = off[lo];
        for (int k = lo; k < hi; ++k) {
            // Givens rotation G(k, k+1) with [c s; -s c]^T [x; z] = [r; 0]
            double c, s;
            if (z == 0.0) {
                c = 1.0;
                s = 0.0;
            } else if (std::fabs(z) > std::fabs(x)) {
                const double t = -x / z;
                s = 1.0 / std::sqrt(1.0 + t * t);
                c = s * t;
            } else {
                const double t = -z / x;
                c = 1.0 / std::sqrt(1.0 + t * t);
                s = c * t;
            }
            // T <- G^T T G on rows/cols k, k+1 (and the bulge at k-1 / k+2)
            if (k > lo) off[k - 1] = c * off[k - 1] - s * z;
            const double a11 = diag[k], a22 = diag[k + 1], a21 = off[k];
            diag[k] = c * c * a11 - 2.0 * c * s * a21 + s * s * a22;
            diag[k + 1] = s * s * a11 + 2.0 * c * s * a21 + c * c * a22;
            off[k] = c * s * (a11 - a22) + (c * c - s * s) * a21;
            if (k + 1 < hi) {
                x = off[k];
                z = -s * off[k + 1];
                off[k + 1] = c * off[k + 1];
            }
            // Q <- Q G: columns k, k+1 (rows k, k+1 of Qt)
            double* qk = &Qt[size_t(k) * d];
            double* qk1 = &Qt[size_t(k + 1) * d];
            for (int i = 0; i < d; ++i) {
                const double u0 = qk[i], u1 = qk1[i];
                qk[i] = c * u0 - s * u1;
                qk1[i] = s * u0 + c * u1;
            }
        }
    }
    for (int i = 0; i < d; ++i) vals[i] = diag[i];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) vecs[size_t(i) * d + j] = Qt[size_t(j) * d + i];
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
