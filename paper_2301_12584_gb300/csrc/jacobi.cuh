// One-CTA symmetric eigendecomposition by cyclic Jacobi (shared by the
// sampler preparation and the pseudo-inverse fallback of the solves).
#pragma once

#include "common.cuh"

namespace krp {

// ---------------------------------------------------------------------------
// One-CTA cyclic Jacobi (Golub & Van Loan, Algorithms 8.5.2-8.5.3, with the
// round-robin ordering of Sec. 8.5.4 so that n/2 disjoint rotations run at
// once).  A (n x n, row-major, symmetric) is overwritten; on exit its diagonal
// holds the eigenvalues and V (n x n) the eigenvectors in its columns.
// Stops when off(A) <= tol ||A||_F, or when a sweep no longer halves off(A)²
// (the off-diagonal mass has reached the rounding floor of Scalar, which for
// FP32 and n ~ 100 lies above 4e-7 ||A||_F; cyclic Jacobi otherwise converges
// quadratically, far faster than that).
// Scalar = float or double.  work: 4 * (n/2 + 1) Scalars, pair: 2*(n/2+1) ints.
// ---------------------------------------------------------------------------
template <typename Scalar>
__device__ void jacobi_eig(Scalar* A, Scalar* V, int n, Scalar* cs, int* pr, double* red,
                           int max_sweeps, double tol) {
    const int m = n + (n & 1);  // players, a dummy when n is odd
    const int npair = m / 2;
    // rotation loops: CH threads per pair, thread (kk, c0) applies pair kk to
    // columns (rows) c0, c0 + CH, ...: the pair's indices and rotation are read
    // once per step, and consecutive threads touch consecutive entries
    const int CH = max(1, (int)blockDim.x / npair);
    const int kk = threadIdx.x / CH, c0 = threadIdx.x % CH;
    const bool has_pair = kk < npair;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = (e / n == e % n) ? Scalar(1) : Scalar(0);
    __syncthreads();
    double off_prev = INFINITY;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // convergence test: off(A)^2 <= tol^2 * ||A||_F^2
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const double a = (double)A[e];
            tot += a * a;
            if (e / n != e % n) off += a * a;
        }
        off = warp_sum_d(off);
        tot = warp_sum_d(tot);
        if ((threadIdx.x & 31) == 0) {
            red[2 * (threadIdx.x >> 5)] = off;
            red[2 * (threadIdx.x >> 5) + 1] = tot;
        }
        __syncthreads();
        double OFF = 0.0, TOT = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            OFF += red[2 * w];
            TOT += red[2 * w + 1];
        }
        __syncthreads();
        if (OFF <= tol * tol * TOT || OFF == 0.0 || (sweep >= 2 && OFF > 0.5 * off_prev)) break;
        off_prev = OFF;
        for (int step = 0; step < m - 1; ++step) {
            for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + step) % (m - 1)) + 1; };
                int p = player(k), q = player(m - 1 - k);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                Scalar c = 1, sn = 0;
                if (q < n) {
                    const Scalar apq = A[p * n + q];
                    if (apq != Scalar(0)) {
                        const Scalar tau = (A[q * n + q] - A[p * n + p]) / (Scalar(2) * apq);
                        const Scalar t = (tau >= Scalar(0) ? Scalar(1) : Scalar(-1)) /
                                         (fabs(tau) + hypot(Scalar(1), tau));
                        c = Scalar(1) / sqrt(Scalar(1) + t * t);
                        sn = t * c;
                    }
                } else {
                    p = -1;
                }
                pr[2 * k] = p;
                pr[2 * k + 1] = q;
                cs[2 * k] = c;
                cs[2 * k + 1] = sn;
            }
            __syncthreads();
            int p = -1, q = 0;
            Scalar c = 1, sn = 0;
            if (has_pair) {
                p = pr[2 * kk];
                q = pr[2 * kk + 1];
                c = cs[2 * kk];
                sn = cs[2 * kk + 1];
            }
            const bool act = p >= 0 && sn != Scalar(0);
            // rows: A <- Jᵀ A
            if (act)
                for (int col = c0; col < n; col += CH) {
                    const Scalar ap = A[p * n + col], aq = A[q * n + col];
                    A[p * n + col] = c * ap - sn * aq;
                    A[q * n + col] = sn * ap + c * aq;
                }
            __syncthreads();
            // columns: A <- A J, V <- V J; the rotated pair's off-diagonal
            // entries (rows p and q) are set to their exact value, zero
            if (act)
                for (int row = c0; row < n; row += CH) {
                    const Scalar ap = A[row * n + p], aq = A[row * n + q];
                    A[row * n + p] = row == q ? Scalar(0) : c * ap - sn * aq;
                    A[row * n + q] = row == p ? Scalar(0) : sn * ap + c * aq;
                    const Scalar vp = V[row * n + p], vq = V[row * n + q];
                    V[row * n + p] = c * vp - sn * vq;
                    V[row * n + q] = sn * vp + c * vq;
                }
            __syncthreads();
        }
    }
}

}  // namespace krp
