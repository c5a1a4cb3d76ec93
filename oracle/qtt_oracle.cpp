// FP64 CPU oracle of the MPS (quantized tensor-train) wave-equation step,
// written in plain C++ with its own Householder QR and one-sided Jacobi SVD:
// no BLAS, no LAPACK, no threads.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, call or
// execute this file or the library built from it; only tests/ do.  It shares
// no code with the CUDA library (paper_2609_01904_b300/csrc) and none with the
// numpy oracle (oracle/qtt_oracle.py): it is a second implementation of the
// same steps, written from the paper, so that the two oracles check each
// other as well as being pinned on their own (tests/test_oracle_cxx.py).
//
// Paper: "Quantum Circuit and Tensor Network Implementation of the 2D
// Acoustic Wave Equation" (Nemeth & Vattay).
//
// Conventions (the readings of the paper are those of the numpy oracle):
//   * dense fields u[x * N + z], N = 2^n, x horizontal, z depth (Sec. 2, Eq. 2);
//   * d = 2n binary sites in the tensor-product order of Eq. 12 (least
//     significant bit first); order 0 = SEQUENTIAL (x register, then z
//     register, Eq. 14-15), order 1 = INTERLEAVED (x_0, z_0, x_1, z_1, ...);
//   * boundary 0 = PERIODIC (the wrap the text states, Sec. 3.1), 1 = ZERO
//     (Eq. 11 as printed: the overflow carry is dropped);
//   * MPS core k: [r_{k-1}][2][r_k], row-major (Eq. 8); MPO core k:
//     [w_{k-1}][t (out)][s (in)][w_k], row-major;
//   * truncation (Sec. 4.3): keep sigma_i >= eps * sigma_1, cap at chi, keep
//     at least one; an all-zero matrix keeps rank 1.
//
// Every function says which passage it follows.  Matrices are row-major.

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Dense matrices and the two factorisations
// ---------------------------------------------------------------------------
struct Mat {
    int m = 0, n = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int rows, int cols) : m(rows), n(cols), a((size_t)rows * cols, 0.0) {}
    double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
    double operator()(int i, int j) const { return a[(size_t)i * n + j]; }
};

Mat transpose(const Mat& A) {
    Mat T(A.n, A.m);
    for (int i = 0; i < A.m; ++i)
        for (int j = 0; j < A.n; ++j) T(j, i) = A(i, j);
    return T;
}

// Thin Householder QR, A (m x n) = Q (m x k) R (k x n), k = min(m, n).
// Reflector j maps column j below the diagonal onto alpha e_1 with alpha of
// the sign opposite to the leading entry (no cancellation); Q is formed by
// applying the reflectors, last first, to the first k columns of I_m
// (Golub & Van Loan, Algorithms 5.1.1-5.1.2 in spirit, written for clarity).
void householder_qr(const Mat& A, Mat& Q, Mat& R) {
    const int m = A.m, n = A.n, k = std::min(m, n);
    Mat W = A;
    std::vector<std::vector<double>> refl(k);
    std::vector<double> vnorm2(k, 0.0);
    for (int j = 0; j < k; ++j) {
        double nx = 0.0;
        for (int i = j; i < m; ++i) nx += W(i, j) * W(i, j);
        nx = std::sqrt(nx);
        std::vector<double> v(m - j);
        for (int i = j; i < m; ++i) v[i - j] = W(i, j);
        const double alpha = v[0] >= 0.0 ? -nx : nx;
        v[0] -= alpha;
        double vv = 0.0;
        for (double x : v) vv += x * x;
        if (vv > 0.0) {
            for (int c = j; c < n; ++c) {
                double dot = 0.0;
                for (int i = j; i < m; ++i) dot += v[i - j] * W(i, c);
                const double f = 2.0 * dot / vv;
                for (int i = j; i < m; ++i) W(i, c) -= f * v[i - j];
            }
        }
        refl[j] = std::move(v);
        vnorm2[j] = vv;
    }
    R = Mat(k, n);
    for (int i = 0; i < k; ++i)
        for (int c = i; c < n; ++c) R(i, c) = W(i, c);
    Q = Mat(m, k);
    for (int i = 0; i < k; ++i) Q(i, i) = 1.0;
    for (int j = k - 1; j >= 0; --j) {
        if (vnorm2[j] == 0.0) continue;
        const std::vector<double>& v = refl[j];
        for (int c = 0; c < k; ++c) {
            double dot = 0.0;
            for (int i = j; i < m; ++i) dot += v[i - j] * Q(i, c);
            const double f = 2.0 * dot / vnorm2[j];
            for (int i = j; i < m; ++i) Q(i, c) -= f * v[i - j];
        }
    }
}

// One-sided Jacobi SVD (Hestenes; de Rijk's cyclic order), M (m x n) =
// U (m x p) diag(S) Vt (p x n), p = min(m, n), S descending.
// Works on the columns of M, or of M^T when M is wide: each pair (p, q) of
// columns is rotated so that the two become orthogonal, with the smaller of
// the two rotation angles, until a whole sweep finds every pair orthogonal
// to m * DBL_EPSILON relative to its norms.  The singular values are the
// final column norms.  Returns the sweep count, or -1 after 80 sweeps.
int jacobi_svd(const Mat& M, Mat& U, std::vector<double>& S, Mat& Vt) {
    const bool wide = M.m < M.n;
    const Mat A = wide ? transpose(M) : M;  // rows >= cols
    const int m = A.m, n = A.n;
    std::vector<std::vector<double>> col(n, std::vector<double>(m));
    std::vector<std::vector<double>> vcol(n, std::vector<double>(n, 0.0));
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < m; ++i) col[j][i] = A(i, j);
        vcol[j][j] = 1.0;
    }
    const double tol = std::max(m, 1) * DBL_EPSILON;
    int sweeps = 0;
    bool converged = (n < 2);
    while (!converged && sweeps < 80) {
        ++sweeps;
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < m; ++i) {
                    alpha += col[p][i] * col[p][i];
                    beta += col[q][i] * col[q][i];
                    gamma += col[p][i] * col[q][i];
                }
                if (gamma == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
                rotated = true;
                // [c_p, c_q] <- [c_p, c_q] [[c, s], [-s, c]] zeroes the cross
                // product when t = s / c solves t^2 + 2 zeta t - 1 = 0.
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < m; ++i) {
                    const double xp = col[p][i], xq = col[q][i];
                    col[p][i] = c * xp - s * xq;
                    col[q][i] = s * xp + c * xq;
                }
                for (int i = 0; i < n; ++i) {
                    const double xp = vcol[p][i], xq = vcol[q][i];
                    vcol[p][i] = c * xp - s * xq;
                    vcol[q][i] = s * xp + c * xq;
                }
            }
        converged = !rotated;
    }
    std::vector<double> norm(n);
    for (int j = 0; j < n; ++j) {
        double s2 = 0.0;
        for (int i = 0; i < m; ++i) s2 += col[j][i] * col[j][i];
        norm[j] = std::sqrt(s2);
    }
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return norm[a] > norm[b]; });
    // left vectors: normalised columns; a zero column is replaced by a unit
    // vector orthogonal to the vectors before it (Gram-Schmidt on e_0, e_1, ...)
    Mat L(m, n), R(n, n);  // A = L diag(S) R^T
    S.assign(n, 0.0);
    for (int jj = 0; jj < n; ++jj) {
        const int j = perm[jj];
        S[jj] = norm[j];
        for (int i = 0; i < n; ++i) R(i, jj) = vcol[j][i];
        if (norm[j] > 0.0) {
            for (int i = 0; i < m; ++i) L(i, jj) = col[j][i] / norm[j];
            continue;
        }
        for (int e = 0; e < m; ++e) {
            std::vector<double> w(m, 0.0);
            w[e] = 1.0;
            for (int kk = 0; kk < jj; ++kk) {
                double dot = 0.0;
                for (int i = 0; i < m; ++i) dot += L(i, kk) * w[i];
                for (int i = 0; i < m; ++i) w[i] -= dot * L(i, kk);
            }
            double wn = 0.0;
            for (double x : w) wn += x * x;
            wn = std::sqrt(wn);
            if (wn > 0.5) {
                for (int i = 0; i < m; ++i) L(i, jj) = w[i] / wn;
                break;
            }
        }
    }
    if (!wide) {  // M = L S R^T
        U = L;
        Vt = transpose(R);
    } else {  // M^T = L S R^T, so M = R S L^T
        U = R;
        Vt = transpose(L);
    }
    return converged ? sweeps : -1;
}

// Sec. 4.3: discard sigma_i < eps * sigma_1, cap at chi, keep at least one.
int trunc_rank(const std::vector<double>& s, double eps, int chi) {
    if (s.empty() || s[0] == 0.0) return 1;
    int r = 0;
    for (double x : s)
        if (x >= eps * s[0]) ++r;
    return std::max(1, std::min(r, chi));
}

// ---------------------------------------------------------------------------
// MPS and MPO containers (Eq. 8; Sec. 4.2)
// ---------------------------------------------------------------------------
struct Core {  // [l][2][r]
    int l = 1, r = 1;
    std::vector<double> a;
    Core() : a(2, 0.0) {}
    Core(int left, int right) : l(left), r(right), a((size_t)left * 2 * right, 0.0) {}
    double& at(int i, int s, int j) { return a[((size_t)i * 2 + s) * r + j]; }
    double at(int i, int s, int j) const { return a[((size_t)i * 2 + s) * r + j]; }
};
using Mps = std::vector<Core>;

struct OpCore {  // [l][t][s][r]
    int l = 1, r = 1;
    std::vector<double> w;
    OpCore(int left, int right) : l(left), r(right), w((size_t)left * 4 * right, 0.0) {}
    double& at(int a, int t, int s, int b) { return w[(((size_t)a * 2 + t) * 2 + s) * r + b]; }
    double at(int a, int t, int s, int b) const { return w[(((size_t)a * 2 + t) * 2 + s) * r + b]; }
};
using Mpo = std::vector<OpCore>;

// ---------------------------------------------------------------------------
// Register encoding (Sec. 3 Eq. 3; Sec. 4.2 Eq. 12, Eq. 14-15)
// ---------------------------------------------------------------------------
// Axis (0 = x, 1 = z) and bit carried by site k.
void site_axis(int n, int order, int k, int& axis, int& bit) {
    if (order == 0) {
        axis = k < n ? 0 : 1;
        bit = k < n ? k : k - n;
    } else {
        axis = k & 1;
        bit = k >> 1;
    }
}

// Flat index of grid point (x, z) in the order-d tensor, site 1 most
// significant (the row-major reshapes of Eq. 8).
int64_t site_index(int n, int order, int x, int z) {
    const int d = 2 * n;
    int64_t idx = 0;
    for (int k = 0; k < d; ++k) {
        int axis, bit;
        site_axis(n, order, k, axis, bit);
        const int s = ((axis == 0 ? x : z) >> bit) & 1;
        idx = idx * 2 + s;
    }
    return idx;
}

// Eq. 8: left-to-right SVDs of the reshaped tensor, each bond truncated by
// the Sec. 4.3 rule.  Cores 1..d-1 come out left-orthonormal.
Mps tt_svd(const std::vector<double>& t, int d, double eps, int chi) {
    Mps cores;
    int r = 1;
    Mat M(1, (int)t.size());
    M.a = t;
    for (int k = 0; k < d - 1; ++k) {
        M.n = (int)(M.a.size() / ((size_t)r * 2));
        M.m = r * 2;
        Mat U, Vt;
        std::vector<double> S;
        jacobi_svd(M, U, S, Vt);
        const int rk = trunc_rank(S, eps, chi);
        Core c(r, rk);
        for (int i = 0; i < r * 2; ++i)
            for (int j = 0; j < rk; ++j) c.a[(size_t)i * rk + j] = U(i, j);
        cores.push_back(std::move(c));
        Mat next(rk, M.n);
        for (int i = 0; i < rk; ++i)
            for (int j = 0; j < M.n; ++j) next(i, j) = S[i] * Vt(i, j);
        M = std::move(next);
        r = rk;
    }
    Core last(r, 1);
    last.a = M.a;
    cores.push_back(std::move(last));
    return cores;
}

Mps mps_from_dense(const double* u, int n, int order, double eps, int chi) {
    const int N = 1 << n, d = 2 * n;
    std::vector<double> t((size_t)1 << d);
    for (int x = 0; x < N; ++x)
        for (int z = 0; z < N; ++z) t[site_index(n, order, x, z)] = u[(size_t)x * N + z];
    return tt_svd(t, d, eps, chi);
}

// Contraction of all cores (Eq. 8 summed over the bonds), site 1 most significant.
std::vector<double> mps_full(const Mps& A) {
    std::vector<double> v(A[0].a);  // (2 x r_1)
    int64_t rows = 2;
    for (size_t k = 1; k < A.size(); ++k) {
        const Core& c = A[k];
        std::vector<double> nv((size_t)rows * 2 * c.r, 0.0);
        for (int64_t i = 0; i < rows; ++i)
            for (int b = 0; b < c.l; ++b) {
                const double x = v[(size_t)i * c.l + b];
                if (x == 0.0) continue;
                for (int s = 0; s < 2; ++s)
                    for (int e = 0; e < c.r; ++e) nv[((size_t)i * 2 + s) * c.r + e] += x * c.at(b, s, e);
            }
        v.swap(nv);
        rows *= 2;
    }
    return v;
}

void mps_to_dense(const Mps& A, int n, int order, double* u) {
    const int N = 1 << n;
    const std::vector<double> t = mps_full(A);
    for (int x = 0; x < N; ++x)
        for (int z = 0; z < N; ++z) u[(size_t)x * N + z] = t[site_index(n, order, x, z)];
}

// u(x, z) = A^(1)_{s_1} ... A^(d)_{s_d} (Eq. 8).
double mps_sample(const Mps& A, int n, int order, int x, int z) {
    std::vector<double> v(1, 1.0);
    for (int k = 0; k < 2 * n; ++k) {
        int axis, bit;
        site_axis(n, order, k, axis, bit);
        const int s = ((axis == 0 ? x : z) >> bit) & 1;
        const Core& c = A[k];
        std::vector<double> nv(c.r, 0.0);
        for (int b = 0; b < c.l; ++b)
            for (int e = 0; e < c.r; ++e) nv[e] += v[b] * c.at(b, s, e);
        v.swap(nv);
    }
    return v[0];
}

// Rank-1 MPS of the unit impulse at (x, z): one-hot cores of its bits.
Mps product_state(int n, int order, int x, int z) {
    Mps out;
    for (int k = 0; k < 2 * n; ++k) {
        int axis, bit;
        site_axis(n, order, k, axis, bit);
        Core c(1, 1);
        c.at(0, ((axis == 0 ? x : z) >> bit) & 1, 0) = 1.0;
        out.push_back(c);
    }
    return out;
}

// ---------------------------------------------------------------------------
// Shift and Laplacian MPOs (Sec. 3.1 Eq. 5-6; Sec. 4.2 Eq. 9-16)
// ---------------------------------------------------------------------------
// 2D shift S_axis^{sign} (Eq. 14-15) in the chosen order.  The bond carries
// the carry (sign +1) or borrow (sign -1) of the increment along the axis'
// bits, least significant first (Eq. 9 / Eq. 13: with no incoming carry the
// bit is copied; with a carry, bit 0 -> 1 absorbs it and bit 1 -> 0 passes
// it on; a borrow the other way round).  The first site of the axis injects
// carry 1 (Eq. 10); sites of the other axis pass the carry through on
// identities; after the axis' last site the outgoing carry is summed over
// (periodic wrap) or only carry 0 is kept (Eq. 11, zero outside the grid).
Mpo shift_mpo(int n, int axis_sel, int sign, int bc, int order) {
    const int d = 2 * n;
    Mpo W;
    int carry_in = 1;  // bond dimension to the left of the current site
    int seen = 0;      // sites of the axis already passed
    for (int k = 0; k < d; ++k) {
        int axis, bit;
        site_axis(n, order, k, axis, bit);
        if (axis != axis_sel) {
            OpCore c(carry_in, carry_in);
            for (int a = 0; a < carry_in; ++a)
                for (int s = 0; s < 2; ++s) c.at(a, s, s, a) = 1.0;
            W.push_back(c);
            continue;
        }
        const bool first = (seen == 0), last = (seen == n - 1);
        ++seen;
        // full carry table T[a_in][t][s][a_out], a in {0, 1}
        double T[2][2][2][2] = {};
        for (int s = 0; s < 2; ++s) T[0][s][s][0] = 1.0;
        if (sign > 0) {
            T[1][1][0][0] = 1.0;  // 0 + carry -> 1, carry absorbed
            T[1][0][1][1] = 1.0;  // 1 + carry -> 0, carry passed on
        } else {
            T[1][0][1][0] = 1.0;  // 1 - borrow -> 0, borrow absorbed
            T[1][1][0][1] = 1.0;  // 0 - borrow -> 1, borrow passed on
        }
        const int lo = first ? 1 : 0, li = first ? 1 : 2;  // incoming: carry 1 only at the first site
        const int ro = last ? 1 : 2;
        OpCore c(li, ro);
        for (int a = 0; a < li; ++a)
            for (int t = 0; t < 2; ++t)
                for (int s = 0; s < 2; ++s)
                    for (int b = 0; b < 2; ++b) {
                        const double v = T[a + lo][t][s][b];
                        if (v == 0.0) continue;
                        if (!last) c.at(a, t, s, b) += v;
                        else if (b == 0 || bc == 0) c.at(a, t, s, 0) += v;
                    }
        W.push_back(c);
        carry_in = ro;
    }
    return W;
}

Mpo identity_mpo(int d) {
    Mpo W;
    for (int k = 0; k < d; ++k) {
        OpCore c(1, 1);
        c.at(0, 0, 0, 0) = c.at(0, 1, 1, 0) = 1.0;
        W.push_back(c);
    }
    return W;
}

// sum_j c_j W_j as one MPO: first cores side by side with the coefficients,
// middle cores block-diagonal, last cores stacked (bonds add up; Sec. 4.3's
// MPS sums written for operators).
Mpo mpo_sum(const std::vector<double>& coef, const std::vector<Mpo>& terms) {
    const size_t d = terms[0].size();
    Mpo out;
    for (size_t k = 0; k < d; ++k) {
        int L = 0, R = 0;
        for (const Mpo& t : terms) {
            L += t[k].l;
            R += t[k].r;
        }
        if (k == 0) L = 1;
        if (k == d - 1) R = 1;
        OpCore c(L, R);
        int lo = 0, ro = 0;
        for (size_t j = 0; j < terms.size(); ++j) {
            const OpCore& b = terms[j][k];
            const double f = (k == 0) ? coef[j] : 1.0;
            for (int a = 0; a < b.l; ++a)
                for (int t = 0; t < 2; ++t)
                    for (int s = 0; s < 2; ++s)
                        for (int e = 0; e < b.r; ++e) c.at(a + lo, t, s, e + ro) += f * b.at(a, t, s, e);
            if (k > 0) lo += b.l;
            if (k < d - 1) ro += b.r;
        }
        out.push_back(c);
    }
    return out;
}

// Eq. 16 as the plain sum of the four lifted shifts and -4I (bond 9); used
// to pin the five-state form below.
Mpo laplacian_sum_of_shifts(int n, int order, int bc) {
    std::vector<Mpo> terms = {shift_mpo(n, 0, +1, bc, order), shift_mpo(n, 0, -1, bc, order),
                              shift_mpo(n, 1, +1, bc, order), shift_mpo(n, 1, -1, bc, order),
                              identity_mpo(2 * n)};
    return mpo_sum({1.0, 1.0, 1.0, 1.0, -4.0}, terms);
}

// Eq. 16 as one carry automaton with five bond states: D (nothing pending,
// identity from here on), XP / XM (an x increment / decrement still
// carrying), ZP / ZM (the same for z).  The left boundary weighs D by -4
// and each shift state by 1 (every shift starts with its carry, Eq. 10); at
// a site of axis a the pending state AP copies nothing: bit 1 -> 0 keeps it
// pending, bit 0 -> 1 resolves it to D; AM the other way round; states of
// the other axis pass by identity, D stays D.  The right boundary accepts
// every state (periodic) or only D (zero, Eq. 11).  Bond states that are
// zero on either side are removed, until no bond shrinks.  This is the
// gauge of the MPO the zip-up truncates in, which the step's result
// depends on.
Mpo laplacian_mpo(int n, int order, int bc) {
    const int d = 2 * n;
    enum { D = 0, XP = 1, XM = 2, ZP = 3, ZM = 4 };
    std::vector<OpCore> W;
    for (int k = 0; k < d; ++k) {
        int axis, bit;
        site_axis(n, order, k, axis, bit);
        OpCore c(5, 5);
        const int p = axis == 0 ? XP : ZP, m = axis == 0 ? XM : ZM;
        const int op = axis == 0 ? ZP : XP, om = axis == 0 ? ZM : XM;
        for (int s = 0; s < 2; ++s) {
            c.at(D, s, s, D) = 1.0;
            c.at(op, s, s, op) = 1.0;
            c.at(om, s, s, om) = 1.0;
        }
        c.at(p, 0, 1, p) = 1.0;  // increment: 1 -> 0, still carrying
        c.at(p, 1, 0, D) = 1.0;  // increment: 0 -> 1, done
        c.at(m, 1, 0, m) = 1.0;  // decrement: 0 -> 1, still borrowing
        c.at(m, 0, 1, D) = 1.0;  // decrement: 1 -> 0, done
        W.push_back(c);
    }
    const double inject[5] = {-4.0, 1.0, 1.0, 1.0, 1.0};
    OpCore first(1, 5);
    for (int a = 0; a < 5; ++a)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s)
                for (int b = 0; b < 5; ++b) first.at(0, t, s, b) += inject[a] * W[0].at(a, t, s, b);
    W[0] = first;
    OpCore lastc(W[d - 1].l, 1);
    for (int a = 0; a < W[d - 1].l; ++a)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s)
                for (int b = 0; b < 5; ++b)
                    if (bc == 0 || b == D) lastc.at(a, t, s, 0) += W[d - 1].at(a, t, s, b);
    W[d - 1] = lastc;
    bool changed = true;
    while (changed) {
        changed = false;
        for (int k = 0; k + 1 < d; ++k) {
            std::vector<int> keep;
            for (int b = 0; b < W[k].r; ++b) {
                bool left_live = false, right_live = false;
                for (int a = 0; a < W[k].l; ++a)
                    for (int t = 0; t < 2; ++t)
                        for (int s = 0; s < 2; ++s) left_live |= W[k].at(a, t, s, b) != 0.0;
                for (int t = 0; t < 2; ++t)
                    for (int s = 0; s < 2; ++s)
                        for (int e = 0; e < W[k + 1].r; ++e) right_live |= W[k + 1].at(b, t, s, e) != 0.0;
                if (left_live && right_live) keep.push_back(b);
            }
            if ((int)keep.size() == W[k].r) continue;
            changed = true;
            OpCore a(W[k].l, (int)keep.size()), b((int)keep.size(), W[k + 1].r);
            for (int x = 0; x < W[k].l; ++x)
                for (int t = 0; t < 2; ++t)
                    for (int s = 0; s < 2; ++s)
                        for (size_t j = 0; j < keep.size(); ++j) a.at(x, t, s, (int)j) = W[k].at(x, t, s, keep[j]);
            for (size_t j = 0; j < keep.size(); ++j)
                for (int t = 0; t < 2; ++t)
                    for (int s = 0; s < 2; ++s)
                        for (int e = 0; e < W[k + 1].r; ++e) b.at((int)j, t, s, e) = W[k + 1].at(keep[j], t, s, e);
            W[k] = a;
            W[k + 1] = b;
        }
    }
    return W;
}

// Sec. 4.3: the diagonal MPO of an MPS, W[r][t][s][r'] = delta_{ts} B[r][s][r'].
Mpo diagonal_mpo(const Mps& B) {
    Mpo W;
    for (const Core& c : B) {
        OpCore w(c.l, c.r);
        for (int a = 0; a < c.l; ++a)
            for (int s = 0; s < 2; ++s)
                for (int b = 0; b < c.r; ++b) w.at(a, s, s, b) = c.at(a, s, b);
        W.push_back(w);
    }
    return W;
}

// ---------------------------------------------------------------------------
// MPS algebra (Sec. 4.3, Eq. 17 and the compression paragraph)
// ---------------------------------------------------------------------------
// Zip-up of W x A from site 1 to site d.  The carried tensor C[a][w][b] (new
// bond, MPO bond, MPS bond) meets core k of the MPS and of the MPO,
//   T[a][t][w'][b'] = sum_{w,s,b} C[a][w][b] A_k[b][s][b'] W_k[w][t][s][w'],
// the matrix T[(a,t)][(w',b')] is split by an SVD, its left vectors (cut by
// the Sec. 4.3 rule) become output core k and S V^T is carried on.
Mps zipup_lr(const Mpo& W, const Mps& A, double eps, int chi) {
    const int d = (int)A.size();
    int ca = 1, cw = 1, cb = 1;
    std::vector<double> C(1, 1.0);  // [ca][cw][cb]
    Mps out;
    for (int k = 0; k < d; ++k) {
        const Core& Ak = A[k];
        const OpCore& Wk = W[k];
        const int wn = Wk.r, bn = Ak.r;
        Mat M(ca * 2, wn * bn);
        for (int a = 0; a < ca; ++a)
            for (int w = 0; w < cw; ++w)
                for (int b = 0; b < cb; ++b) {
                    const double x = C[((size_t)a * cw + w) * cb + b];
                    if (x == 0.0) continue;
                    for (int s = 0; s < 2; ++s)
                        for (int e = 0; e < bn; ++e) {
                            const double y = x * Ak.at(b, s, e);
                            if (y == 0.0) continue;
                            for (int t = 0; t < 2; ++t)
                                for (int v = 0; v < wn; ++v) M(a * 2 + t, v * bn + e) += y * Wk.at(w, t, s, v);
                        }
                }
        if (k == d - 1) {
            Core c(ca, 1);
            c.a = M.a;
            out.push_back(std::move(c));
            break;
        }
        Mat U, Vt;
        std::vector<double> S;
        jacobi_svd(M, U, S, Vt);
        const int r = trunc_rank(S, eps, chi);
        Core c(ca, r);
        for (int i = 0; i < ca * 2; ++i)
            for (int j = 0; j < r; ++j) c.a[(size_t)i * r + j] = U(i, j);
        out.push_back(std::move(c));
        C.assign((size_t)r * wn * bn, 0.0);
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < wn * bn; ++j) C[(size_t)i * wn * bn + j] = S[i] * Vt(i, j);
        ca = r;
        cw = wn;
        cb = bn;
    }
    return out;
}

// Mirror of zipup_lr from site d to site 1:
//   T[b][w][t][a'] = sum_{s,b',w'} A_k[b][s][b'] W_k[w][t][s][w'] C[b'][w'][a'],
// the matrix T[(b,w)][(t,a')] is split by an SVD, its right vectors become
// output core k and U S is carried on.
Mps zipup_rl(const Mpo& W, const Mps& A, double eps, int chi) {
    const int d = (int)A.size();
    int cb = 1, cw = 1, ca = 1;
    std::vector<double> C(1, 1.0);  // [cb][cw][ca]
    Mps out(d);
    for (int k = d - 1; k >= 0; --k) {
        const Core& Ak = A[k];
        const OpCore& Wk = W[k];
        const int bn = Ak.l, wn = Wk.l;
        Mat M(bn * wn, 2 * ca);
        for (int b = 0; b < bn; ++b)
            for (int s = 0; s < 2; ++s)
                for (int e = 0; e < cb; ++e) {
                    const double x = Ak.at(b, s, e);
                    if (x == 0.0) continue;
                    for (int w = 0; w < wn; ++w)
                        for (int t = 0; t < 2; ++t)
                            for (int v = 0; v < cw; ++v) {
                                const double y = x * Wk.at(w, t, s, v);
                                if (y == 0.0) continue;
                                for (int a = 0; a < ca; ++a) M(b * wn + w, t * ca + a) += y * C[((size_t)e * cw + v) * ca + a];
                            }
                }
        if (k == 0) {
            Core c(1, ca);
            c.a = M.a;
            out[0] = std::move(c);
            break;
        }
        Mat U, Vt;
        std::vector<double> S;
        jacobi_svd(M, U, S, Vt);
        const int r = trunc_rank(S, eps, chi);
        Core c(r, ca);
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < 2 * ca; ++j) c.a[(size_t)i * 2 * ca + j] = Vt(i, j);
        out[k] = std::move(c);
        C.assign((size_t)bn * wn * r, 0.0);
        for (int i = 0; i < bn * wn; ++i)
            for (int j = 0; j < r; ++j) C[(size_t)i * r + j] = U(i, j) * S[j];
        cb = bn;
        cw = wn;
        ca = r;
    }
    return out;
}

// sum_j c_j |psi_j> as one MPS (Sec. 4.3): first cores side by side with the
// coefficients folded in, middle cores block-diagonal, last cores stacked.
Mps mps_sum(const std::vector<double>& coef, const std::vector<const Mps*>& terms) {
    const size_t d = terms[0]->size();
    Mps out;
    for (size_t k = 0; k < d; ++k) {
        int L = 0, R = 0;
        for (const Mps* t : terms) {
            L += (*t)[k].l;
            R += (*t)[k].r;
        }
        if (k == 0) L = 1;
        if (k == d - 1) R = 1;
        Core c(L, R);
        int lo = 0, ro = 0;
        for (size_t j = 0; j < terms.size(); ++j) {
            const Core& b = (*terms[j])[k];
            const double f = (k == 0) ? coef[j] : 1.0;
            for (int a = 0; a < b.l; ++a)
                for (int s = 0; s < 2; ++s)
                    for (int e = 0; e < b.r; ++e) c.at(a + lo, s, e + ro) += f * b.at(a, s, e);
            if (k > 0) lo += b.l;
            if (k < d - 1) ro += b.r;
        }
        out.push_back(std::move(c));
    }
    return out;
}

// Compression (Sec. 4.3): left-to-right QR sweep (core k = Q, R moves into
// core k+1), then right-to-left SVD sweep truncating every bond by the rule.
Mps tt_round(Mps A, double eps, int chi) {
    const int d = (int)A.size();
    for (int k = 0; k + 1 < d; ++k) {
        Mat M(A[k].l * 2, A[k].r);
        M.a = A[k].a;
        Mat Q, R;
        householder_qr(M, Q, R);
        const int kk = Q.n;
        Core q(A[k].l, kk);
        q.a = Q.a;
        const Core& nx = A[k + 1];
        Core nn(kk, nx.r);
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < nx.l; ++j) {
                const double rij = R(i, j);
                if (rij == 0.0) continue;
                for (int s = 0; s < 2; ++s)
                    for (int e = 0; e < nx.r; ++e) nn.at(i, s, e) += rij * nx.at(j, s, e);
            }
        A[k] = std::move(q);
        A[k + 1] = std::move(nn);
    }
    for (int k = d - 1; k > 0; --k) {
        Mat M(A[k].l, 2 * A[k].r);
        M.a = A[k].a;
        Mat U, Vt;
        std::vector<double> S;
        jacobi_svd(M, U, S, Vt);
        const int rr = trunc_rank(S, eps, chi);
        Core v(rr, A[k].r);
        for (int i = 0; i < rr; ++i)
            for (int j = 0; j < 2 * A[k].r; ++j) v.a[(size_t)i * 2 * A[k].r + j] = Vt(i, j);
        const Core& pv = A[k - 1];
        Core np(pv.l, rr);
        for (int a = 0; a < pv.l; ++a)
            for (int s = 0; s < 2; ++s)
                for (int j = 0; j < pv.r; ++j) {
                    const double x = pv.at(a, s, j);
                    if (x == 0.0) continue;
                    for (int e = 0; e < rr; ++e) np.at(a, s, e) += x * U(j, e) * S[e];
                }
        A[k] = std::move(v);
        A[k - 1] = std::move(np);
    }
    return A;
}

// One time step of Eq. 17 in MPS form:
//   phi = L psi^k (zip-up, sites 1 -> d); eta = C^2 phi (zip-up of diag(c^2),
//   sites d -> 1); theta = 2 psi^k - psi^{k-1} + lambda^2 eta [+ amp e_src];
//   psi^{k+1} = round(theta).
Mps mps_step(const Mpo& L, const Mps& c2, double lambda2, const Mps& prev, const Mps& cur, double eps, int chi,
             int sx, int sz, double amp, int n, int order) {
    const Mps phi = zipup_lr(L, cur, eps, chi);
    const Mps eta = zipup_rl(diagonal_mpo(c2), phi, eps, chi);
    std::vector<double> coef = {2.0, -1.0, lambda2};
    std::vector<const Mps*> terms = {&cur, &prev, &eta};
    Mps src;
    if (sx >= 0) {
        src = product_state(n, order, sx, sz);
        coef.push_back(amp);
        terms.push_back(&src);
    }
    return tt_round(mps_sum(coef, terms), eps, chi);
}

// Operator matrix of an MPO on the dense grid, out[(x N + z) * N^2 + (x' N + z')].
void mpo_grid_operator(const Mpo& W, int n, int order, double* out) {
    const int N = 1 << n, d = 2 * n;
    const int64_t NN = (int64_t)N * N;
    for (int64_t p = 0; p < NN; ++p)
        for (int64_t q = 0; q < NN; ++q) {
            const int xo = (int)(p / N), zo = (int)(p % N), xi = (int)(q / N), zi = (int)(q % N);
            std::vector<double> v(1, 1.0);
            for (int k = 0; k < d && !v.empty(); ++k) {
                int axis, bit;
                site_axis(n, order, k, axis, bit);
                const int t = ((axis == 0 ? xo : zo) >> bit) & 1, s = ((axis == 0 ? xi : zi) >> bit) & 1;
                std::vector<double> nv(W[k].r, 0.0);
                for (int a = 0; a < W[k].l; ++a)
                    for (int b = 0; b < W[k].r; ++b) nv[b] += v[a] * W[k].at(a, t, s, b);
                v.swap(nv);
            }
            out[p * NN + q] = v[0];
        }
}

// ---------------------------------------------------------------------------
// Dense FDTD (Sec. 2, Eq. 2)
// ---------------------------------------------------------------------------
void fdtd_step(int N, const double* prev, const double* cur, const double* c2, double lambda2, int bc, int sx, int sz,
               double amp, double* out) {
    auto at = [&](int x, int z) -> double {
        if (bc == 0) return cur[(size_t)((x + N) % N) * N + (z + N) % N];
        if (x < 0 || x >= N || z < 0 || z >= N) return 0.0;
        return cur[(size_t)x * N + z];
    };
    for (int x = 0; x < N; ++x)
        for (int z = 0; z < N; ++z) {
            const size_t i = (size_t)x * N + z;
            const double lap = at(x + 1, z) + at(x - 1, z) + at(x, z + 1) + at(x, z - 1) - 4.0 * cur[i];
            out[i] = 2.0 * cur[i] - prev[i] + lambda2 * c2[i] * lap;
        }
    if (sx >= 0) out[(size_t)sx * N + sz] += amp;
}

Mps* box(Mps&& m) { return new Mps(std::move(m)); }
Mpo* box(Mpo&& m) { return new Mpo(std::move(m)); }

}  // namespace

// ---------------------------------------------------------------------------
// C interface for the tests (ctypes).  Handles own their cores; every call
// that returns a handle returns a new one.  No call throws or exits.
// ---------------------------------------------------------------------------
extern "C" {

void* oc_mps_from_cores(int d, const int* ranks, const double* data) {
    Mps A;
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
        Core c(ranks[k], ranks[k + 1]);
        std::memcpy(c.a.data(), data + off, c.a.size() * sizeof(double));
        off += c.a.size();
        A.push_back(std::move(c));
    }
    return box(std::move(A));
}
int oc_mps_sites(const void* h) { return (int)static_cast<const Mps*>(h)->size(); }
void oc_mps_ranks(const void* h, int* ranks) {
    const Mps& A = *static_cast<const Mps*>(h);
    ranks[0] = A.empty() ? 1 : A[0].l;
    for (size_t k = 0; k < A.size(); ++k) ranks[k + 1] = A[k].r;
}
void oc_mps_data(const void* h, double* out) {
    for (const Core& c : *static_cast<const Mps*>(h)) {
        std::memcpy(out, c.a.data(), c.a.size() * sizeof(double));
        out += c.a.size();
    }
}
void oc_mps_free(void* h) { delete static_cast<Mps*>(h); }

void* oc_mps_from_dense(int n, int order, const double* u, double eps, int chi) {
    return box(mps_from_dense(u, n, order, eps, chi));
}
void oc_mps_to_dense(const void* h, int n, int order, double* u) { mps_to_dense(*static_cast<const Mps*>(h), n, order, u); }
void oc_mps_sample(const void* h, int n, int order, int np, const int* ix, const int* iz, double* out) {
    for (int p = 0; p < np; ++p) out[p] = mps_sample(*static_cast<const Mps*>(h), n, order, ix[p], iz[p]);
}
void* oc_product_state(int n, int order, int x, int z) { return box(product_state(n, order, x, z)); }
void* oc_round(const void* h, double eps, int chi) { return box(tt_round(*static_cast<const Mps*>(h), eps, chi)); }
void* oc_sum(int nterms, const double* coef, void* const* terms) {
    std::vector<double> c(coef, coef + nterms);
    std::vector<const Mps*> t;
    for (int j = 0; j < nterms; ++j) t.push_back(static_cast<const Mps*>(terms[j]));
    return box(mps_sum(c, t));
}

void* oc_shift_mpo(int n, int axis, int sign, int bc, int order) { return box(shift_mpo(n, axis, sign, bc, order)); }
void* oc_laplacian_mpo(int n, int order, int bc) { return box(laplacian_mpo(n, order, bc)); }
void* oc_laplacian_sum_of_shifts(int n, int order, int bc) { return box(laplacian_sum_of_shifts(n, order, bc)); }
void* oc_diagonal_mpo(const void* h) { return box(diagonal_mpo(*static_cast<const Mps*>(h))); }
int oc_mpo_sites(const void* h) { return (int)static_cast<const Mpo*>(h)->size(); }
void oc_mpo_bonds(const void* h, int* bonds) {
    const Mpo& W = *static_cast<const Mpo*>(h);
    bonds[0] = W.empty() ? 1 : W[0].l;
    for (size_t k = 0; k < W.size(); ++k) bonds[k + 1] = W[k].r;
}
void oc_mpo_data(const void* h, double* out) {
    for (const OpCore& c : *static_cast<const Mpo*>(h)) {
        std::memcpy(out, c.w.data(), c.w.size() * sizeof(double));
        out += c.w.size();
    }
}
void oc_mpo_grid_operator(const void* h, int n, int order, double* out) {
    mpo_grid_operator(*static_cast<const Mpo*>(h), n, order, out);
}
void oc_mpo_free(void* h) { delete static_cast<Mpo*>(h); }

void* oc_zipup_lr(const void* W, const void* A, double eps, int chi) {
    return box(zipup_lr(*static_cast<const Mpo*>(W), *static_cast<const Mps*>(A), eps, chi));
}
void* oc_zipup_rl(const void* W, const void* A, double eps, int chi) {
    return box(zipup_rl(*static_cast<const Mpo*>(W), *static_cast<const Mps*>(A), eps, chi));
}
void* oc_step(const void* L, const void* c2, double lambda2, const void* prev, const void* cur, double eps, int chi,
              int sx, int sz, double amp, int n, int order) {
    return box(mps_step(*static_cast<const Mpo*>(L), *static_cast<const Mps*>(c2), lambda2,
                        *static_cast<const Mps*>(prev), *static_cast<const Mps*>(cur), eps, chi, sx, sz, amp, n, order));
}
void oc_fdtd_step(int N, const double* prev, const double* cur, const double* c2, double lambda2, int bc, int sx,
                  int sz, double amp, double* out) {
    fdtd_step(N, prev, cur, c2, lambda2, bc, sx, sz, amp, out);
}

// M (m x n) = U (m x p) diag(S) Vt (p x n), p = min(m, n); returns the sweep
// count or -1 when the sweep limit was reached.
int oc_svd(int m, int n, const double* M, double* U, double* S, double* Vt) {
    Mat A(m, n);
    std::memcpy(A.a.data(), M, A.a.size() * sizeof(double));
    Mat u, vt;
    std::vector<double> s;
    const int sweeps = jacobi_svd(A, u, s, vt);
    std::memcpy(U, u.a.data(), u.a.size() * sizeof(double));
    std::memcpy(S, s.data(), s.size() * sizeof(double));
    std::memcpy(Vt, vt.a.data(), vt.a.size() * sizeof(double));
    return sweeps;
}

// A (m x n) = Q (m x k) R (k x n), k = min(m, n).
void oc_qr(int m, int n, const double* A, double* Q, double* R) {
    Mat a(m, n);
    std::memcpy(a.a.data(), A, a.a.size() * sizeof(double));
    Mat q, r;
    householder_qr(a, q, r);
    std::memcpy(Q, q.a.data(), q.a.size() * sizeof(double));
    std::memcpy(R, r.a.data(), r.a.size() * sizeof(double));
}

int oc_trunc_rank(int p, const double* s, double eps, int chi) {
    return trunc_rank(std::vector<double>(s, s + p), eps, chi);
}

}  // extern "C"
