/*
 * CPU oracle for the implicit distance-matrix product (Indyk & Silwal,
 * "Faster Linear Algebra for Distance Matrices", arXiv 2210.15114).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file: it is used by the tests, by the package's smoke check and
 * by the benchmark's CPU-baseline leg.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Everything here is the plain definition of the product, written out as a
 * direct double loop:
 *
 *     (A Z)[r, :] = sum_j f(x_r, x_j) * Z[j, :]
 *
 * with f = ||x - y||_1 (Section 2, the matrix A_ij = ||x_i - x_j||_1 used by
 * Theorem "p=1") or f = ||x - y||_2^2 (Appendix A, Theorem for p = 2).
 * Rows are evaluated one at a time, so the caller can ask for a sample of
 * rows of a large product (each row costs O(n d k)).  The same file holds the
 * gradient of w^T A(X) z with respect to X (end of file), also as a direct
 * double loop.
 *
 * Floating point is FP64 with the terms summed in index order j = 0..n-1.
 * The integer forms use int64 arithmetic; two's-complement wrap-around makes
 * the final value exact whenever the true result fits in int64.
 *
 * Layout: X is n x d row-major (point j is row j), Z is n x k row-major,
 * out is nrows x k row-major, rows[] lists the row indices to evaluate.
 */
#include <stdint.h>
#include <math.h>

/* |a - b| for int64 without relying on a library call. */
static int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

/* l1 product, FP64: out[r,:] = sum_j ||x_rows[r] - x_j||_1 Z[j,:]. */
void oracle_l1_rows_f64(const double* X, int64_t n, int64_t d,
                        const double* Z, int64_t k,
                        const int64_t* rows, int64_t nrows, double* out) {
    for (int64_t r = 0; r < nrows; ++r) {
        const double* xr = X + rows[r] * d;
        double* o = out + r * k;
        for (int64_t c = 0; c < k; ++c) o[c] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double* xj = X + j * d;
            double dist = 0.0;
            for (int64_t i = 0; i < d; ++i) dist += fabs(xr[i] - xj[i]);
            const double* zj = Z + j * k;
            for (int64_t c = 0; c < k; ++c) o[c] += dist * zj[c];
        }
    }
}

/* squared-l2 product, FP64: out[r,:] = sum_j ||x_rows[r] - x_j||_2^2 Z[j,:]. */
void oracle_l2sq_rows_f64(const double* X, int64_t n, int64_t d,
                          const double* Z, int64_t k,
                          const int64_t* rows, int64_t nrows, double* out) {
    for (int64_t r = 0; r < nrows; ++r) {
        const double* xr = X + rows[r] * d;
        double* o = out + r * k;
        for (int64_t c = 0; c < k; ++c) o[c] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double* xj = X + j * d;
            double dist = 0.0;
            for (int64_t i = 0; i < d; ++i) {
                double t = xr[i] - xj[i];
                dist += t * t;
            }
            const double* zj = Z + j * k;
            for (int64_t c = 0; c < k; ++c) o[c] += dist * zj[c];
        }
    }
}

/* l1 product, exact integers (int64 coordinates and weights). */
void oracle_l1_rows_i64(const int64_t* X, int64_t n, int64_t d,
                        const int64_t* Z, int64_t k,
                        const int64_t* rows, int64_t nrows, int64_t* out) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t* xr = X + rows[r] * d;
        int64_t* o = out + r * k;
        for (int64_t c = 0; c < k; ++c) o[c] = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t* xj = X + j * d;
            int64_t dist = 0;
            for (int64_t i = 0; i < d; ++i) dist += iabs64(xr[i] - xj[i]);
            const int64_t* zj = Z + j * k;
            for (int64_t c = 0; c < k; ++c)
                o[c] = (int64_t)((uint64_t)o[c] + (uint64_t)dist * (uint64_t)zj[c]);
        }
    }
}

/* squared-l2 product, exact integers (int64 coordinates and weights). */
void oracle_l2sq_rows_i64(const int64_t* X, int64_t n, int64_t d,
                          const int64_t* Z, int64_t k,
                          const int64_t* rows, int64_t nrows, int64_t* out) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t* xr = X + rows[r] * d;
        int64_t* o = out + r * k;
        for (int64_t c = 0; c < k; ++c) o[c] = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t* xj = X + j * d;
            int64_t dist = 0;
            for (int64_t i = 0; i < d; ++i) {
                int64_t t = xr[i] - xj[i];
                dist += t * t;
            }
            const int64_t* zj = Z + j * k;
            for (int64_t c = 0; c < k; ++c)
                o[c] = (int64_t)((uint64_t)o[c] + (uint64_t)dist * (uint64_t)zj[c]);
        }
    }
}

/*
 * Gradient of L = sum_q w_q^T A(X) z_q with respect to the points X (k pairs
 * of columns w_q, z_q of W and Z).  The paper states no gradient; this is the
 * chain rule applied to the definition.  Only the terms with a = i or b = i
 * of L = sum_a sum_b w_a z_b f(x_a, x_b) depend on x_i, and f is a sum over
 * coordinates of phi(x(c) - y(c)) with phi even, so
 *
 *     dL/dx_i(c) = sum_q sum_j (w[i,q] z[j,q] + z[i,q] w[j,q]) phi'(x_i(c) - x_j(c))
 *
 * with phi' = sgn (and sgn(0) = 0, the symmetric subgradient) for l1 and
 * phi'(t) = 2 t for squared l2.  G is nrows x d row-major, one row per
 * requested point.  W and Z are n x k row-major.
 */
static double sgn_f64(double t) { return t > 0.0 ? 1.0 : (t < 0.0 ? -1.0 : 0.0); }
static int64_t sgn_i64(int64_t t) { return t > 0 ? 1 : (t < 0 ? -1 : 0); }

void oracle_l1_grad_rows_f64(const double* X, int64_t n, int64_t d,
                             const double* W, const double* Z, int64_t k,
                             const int64_t* rows, int64_t nrows, double* G) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        const double* xi = X + i * d;
        double* g = G + r * d;
        for (int64_t c = 0; c < d; ++c) g[c] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double* xj = X + j * d;
            double weight = 0.0;
            for (int64_t q = 0; q < k; ++q)
                weight += W[i * k + q] * Z[j * k + q] + Z[i * k + q] * W[j * k + q];
            for (int64_t c = 0; c < d; ++c) g[c] += weight * sgn_f64(xi[c] - xj[c]);
        }
    }
}

void oracle_l2sq_grad_rows_f64(const double* X, int64_t n, int64_t d,
                               const double* W, const double* Z, int64_t k,
                               const int64_t* rows, int64_t nrows, double* G) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        const double* xi = X + i * d;
        double* g = G + r * d;
        for (int64_t c = 0; c < d; ++c) g[c] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double* xj = X + j * d;
            double weight = 0.0;
            for (int64_t q = 0; q < k; ++q)
                weight += W[i * k + q] * Z[j * k + q] + Z[i * k + q] * W[j * k + q];
            for (int64_t c = 0; c < d; ++c) g[c] += weight * (2.0 * (xi[c] - xj[c]));
        }
    }
}

/* The same two gradients in exact integer arithmetic (int64 wrap-around is
 * exact whenever the true result fits in int64). */
void oracle_l1_grad_rows_i64(const int64_t* X, int64_t n, int64_t d,
                             const int64_t* W, const int64_t* Z, int64_t k,
                             const int64_t* rows, int64_t nrows, int64_t* G) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        const int64_t* xi = X + i * d;
        int64_t* g = G + r * d;
        for (int64_t c = 0; c < d; ++c) g[c] = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t* xj = X + j * d;
            uint64_t weight = 0;
            for (int64_t q = 0; q < k; ++q)
                weight += (uint64_t)W[i * k + q] * (uint64_t)Z[j * k + q] +
                          (uint64_t)Z[i * k + q] * (uint64_t)W[j * k + q];
            for (int64_t c = 0; c < d; ++c)
                g[c] = (int64_t)((uint64_t)g[c] + weight * (uint64_t)sgn_i64(xi[c] - xj[c]));
        }
    }
}

void oracle_l2sq_grad_rows_i64(const int64_t* X, int64_t n, int64_t d,
                               const int64_t* W, const int64_t* Z, int64_t k,
                               const int64_t* rows, int64_t nrows, int64_t* G) {
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        const int64_t* xi = X + i * d;
        int64_t* g = G + r * d;
        for (int64_t c = 0; c < d; ++c) g[c] = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t* xj = X + j * d;
            uint64_t weight = 0;
            for (int64_t q = 0; q < k; ++q)
                weight += (uint64_t)W[i * k + q] * (uint64_t)Z[j * k + q] +
                          (uint64_t)Z[i * k + q] * (uint64_t)W[j * k + q];
            for (int64_t c = 0; c < d; ++c)
                g[c] = (int64_t)((uint64_t)g[c] + weight * (uint64_t)(2 * (xi[c] - xj[c])));
        }
    }
}
