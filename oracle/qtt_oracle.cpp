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
// Besides the 2D step it covers the transition operator of Eq. 7 as one
// MPO and the fused step, the 3D extension of Sec. 6 (three registers, the
// 7-point Laplacian), and the learned form (rank features, the MLP with
// its gradient and Adam, the randomised range finder with its exact
// acceptance check, the round that uses it; oracle/cxx_learned.py).  Every
// function is pinned by tests/test_oracle_cxx.py, tests/test_oracle_learned.py
// or tests/test_oracle_symmetry.py.
//
// Conventions (the readings of the paper are those of the numpy oracle):
//   * dense fields u[x * N + z], N = 2^n, x horizontal, z depth (Sec. 2,
//     Eq. 2); in 3D u[(x * N + y) * N + z];
//   * d = dims * n binary sites in the tensor-product order of Eq. 12 (least
//     significant bit first); order 0 = SEQUENTIAL (one register after the
//     other, Eq. 14-15), order 1 = INTERLEAVED (x_0, z_0, x_1, z_1, ...; in
//     3D x_0, y_0, z_0, x_1, ...);
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
// The reflector is built from the column divided by its largest entry (the
// reflection depends only on the direction): squares of entries near the
// underflow threshold would otherwise vanish and leave it non-orthogonal.
// A column with nothing below the diagonal is left as it is (identity, not
// a sign flip), the convention of the common LAPACK-style QR, so that the
// two oracles put the bonds in the same gauge: the randomised range finder
// of the learned form sketches in that gauge.
void householder_qr(const Mat& A, Mat& Q, Mat& R) {
    const int m = A.m, n = A.n, k = std::min(m, n);
    Mat W = A;
    std::vector<std::vector<double>> refl(k);
    std::vector<double> vnorm2(k, 0.0);
    for (int j = 0; j < k; ++j) {
        double sc = 0.0, below = 0.0;
        for (int i = j; i < m; ++i) sc = std::max(sc, std::fabs(W(i, j)));
        for (int i = j + 1; i < m; ++i) below = std::max(below, std::fabs(W(i, j)));
        std::vector<double> v(m - j, 0.0);
        if (below == 0.0) {  // nothing below the diagonal to annihilate: identity
            refl[j] = std::move(v);
            continue;
        }
        double nx = 0.0;
        for (int i = j; i < m; ++i) {
            v[i - j] = W(i, j) / sc;
            nx += v[i - j] * v[i - j];
        }
        nx = std::sqrt(nx);
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

// Euclidean norm of x[0..m) computed on x / max|x_i|, so that squares of
// entries near the underflow (or overflow) threshold do not vanish (blow up).
double norm_scaled(const std::vector<double>& x) {
    double sc = 0.0;
    for (double v : x) sc = std::max(sc, std::fabs(v));
    if (sc == 0.0) return 0.0;
    double s2 = 0.0;
    for (double v : x) s2 += (v / sc) * (v / sc);
    return sc * std::sqrt(s2);
}

// One-sided Jacobi SVD (Hestenes; de Rijk's cyclic order), M (m x n) =
// U (m x p) diag(S) Vt (p x n), p = min(m, n), S descending.
// Works on the columns of M, or of M^T when M is wide: each pair (p, q) of
// columns is rotated so that the two become orthogonal, with the smaller of
// the two rotation angles, until a whole sweep finds every pair orthogonal
// to m * DBL_EPSILON (the cosine of the angle between them, computed on the
// normalised columns).  A rotation too small to change a column in FP64 is
// not counted.  The singular values are the final column norms.  Returns
// the sweep count, or -1 after 80 sweeps.
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
                const double np_ = norm_scaled(col[p]), nq_ = norm_scaled(col[q]);
                if (np_ == 0.0 || nq_ == 0.0) continue;
                double rho = 0.0;  // cosine of the angle between the two columns
                for (int i = 0; i < m; ++i) rho += (col[p][i] / np_) * (col[q][i] / nq_);
                if (std::fabs(rho) <= tol) continue;
                // [c_p, c_q] <- [c_p, c_q] [[c, s], [-s, c]] zeroes the cross
                // product when t = s / c solves t^2 + 2 zeta t - 1 = 0, with
                // zeta = (|c_q|^2 - |c_p|^2) / (2 c_p . c_q)
                const double zeta = (nq_ / np_ - np_ / nq_) / (2.0 * rho);
                // (hypot: zeta reaches 1e160 and more for columns of very different size)
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::hypot(1.0, zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                if (s == 0.0) continue;
                rotated = true;
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
    for (int j = 0; j < n; ++j) norm[j] = norm_scaled(col[j]);
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
// A grid of dims axes (2: x, z; 3: x, y, z for the extension of Sec. 6),
// N = 2^n points per axis, d = dims * n sites.  Dense fields are indexed by
// the point's coordinates in axis order, the last fastest: u[x N + z] in 2D,
// u[(x N + y) N + z] in 3D.
struct Grid {
    int dims = 2, n = 1, order = 1;
    int d() const { return dims * n; }
    int N() const { return 1 << n; }
    int64_t points() const { return (int64_t)1 << (dims * n); }
};

// Axis and bit carried by site k: least significant bit first per axis
// (Eq. 12); SEQUENTIAL puts the registers one after another (Eq. 14-15),
// INTERLEAVED takes bit b of every axis before bit b+1.
void site_axis(const Grid& g, int k, int& axis, int& bit) {
    if (g.order == 0) {
        axis = k / g.n;
        bit = k % g.n;
    } else {
        axis = k % g.dims;
        bit = k / g.dims;
    }
}

// Coordinates of the point with dense index lin.
void coords(const Grid& g, int64_t lin, int* p) {
    for (int a = g.dims - 1; a >= 0; --a) {
        p[a] = (int)(lin % g.N());
        lin /= g.N();
    }
}

// Flat index of a point in the order-d tensor, site 1 most significant (the
// row-major reshapes of Eq. 8).
int64_t site_index(const Grid& g, const int* p) {
    int64_t idx = 0;
    for (int k = 0; k < g.d(); ++k) {
        int axis, bit;
        site_axis(g, k, axis, bit);
        idx = idx * 2 + ((p[axis] >> bit) & 1);
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

Mps mps_from_dense(const Grid& g, const double* u, double eps, int chi) {
    std::vector<double> t((size_t)g.points());
    int p[3];
    for (int64_t lin = 0; lin < g.points(); ++lin) {
        coords(g, lin, p);
        t[site_index(g, p)] = u[lin];
    }
    return tt_svd(t, g.d(), eps, chi);
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

void mps_to_dense(const Grid& g, const Mps& A, double* u) {
    const std::vector<double> t = mps_full(A);
    int p[3];
    for (int64_t lin = 0; lin < g.points(); ++lin) {
        coords(g, lin, p);
        u[lin] = t[site_index(g, p)];
    }
}

// u(p) = A^(1)_{s_1} ... A^(d)_{s_d} (Eq. 8).
double mps_sample(const Grid& g, const Mps& A, const int* p) {
    std::vector<double> v(1, 1.0);
    for (int k = 0; k < g.d(); ++k) {
        int axis, bit;
        site_axis(g, k, axis, bit);
        const int s = (p[axis] >> bit) & 1;
        const Core& c = A[k];
        std::vector<double> nv(c.r, 0.0);
        for (int b = 0; b < c.l; ++b)
            for (int e = 0; e < c.r; ++e) nv[e] += v[b] * c.at(b, s, e);
        v.swap(nv);
    }
    return v[0];
}

// Rank-1 MPS of the unit impulse at p: one-hot cores of its bits.
Mps product_state(const Grid& g, const int* p) {
    Mps out;
    for (int k = 0; k < g.d(); ++k) {
        int axis, bit;
        site_axis(g, k, axis, bit);
        Core c(1, 1);
        c.at(0, (p[axis] >> bit) & 1, 0) = 1.0;
        out.push_back(c);
    }
    return out;
}

// ---------------------------------------------------------------------------
// Shift and Laplacian MPOs (Sec. 3.1 Eq. 5-6; Sec. 4.2 Eq. 9-16)
// ---------------------------------------------------------------------------
// Shift S_axis^{sign} lifted to the grid (Eq. 14-15).  The bond carries the
// carry (sign +1) or borrow (sign -1) of the increment along the axis' bits,
// least significant first (Eq. 9 / Eq. 13: with no incoming carry the bit
// is copied; with a carry, bit 0 -> 1 absorbs it and bit 1 -> 0 passes it
// on; a borrow the other way round).  The first site of the axis injects
// carry 1 (Eq. 10); sites of other axes pass the carry through on
// identities; after the axis' last site the outgoing carry is summed over
// (periodic wrap) or only carry 0 is kept (Eq. 11, zero outside the grid).
Mpo shift_mpo(const Grid& g, int axis_sel, int sign, int bc) {
    Mpo W;
    int carry_in = 1;  // bond dimension to the left of the current site
    int seen = 0;      // sites of the axis already passed
    for (int k = 0; k < g.d(); ++k) {
        int axis, bit;
        site_axis(g, k, axis, bit);
        if (axis != axis_sel) {
            OpCore c(carry_in, carry_in);
            for (int a = 0; a < carry_in; ++a)
                for (int s = 0; s < 2; ++s) c.at(a, s, s, a) = 1.0;
            W.push_back(c);
            continue;
        }
        const bool first = (seen == 0), last = (seen == g.n - 1);
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

// Eq. 16 (Eq. 6 with a third pair of shifts in 3D) as the plain sum of the
// lifted shifts and -2 dims I (bond 4 dims + 1); used to pin the automaton.
Mpo laplacian_sum_of_shifts(const Grid& g, int bc) {
    std::vector<Mpo> terms;
    std::vector<double> coef;
    for (int a = 0; a < g.dims; ++a)
        for (int sign : {+1, -1}) {
            terms.push_back(shift_mpo(g, a, sign, bc));
            coef.push_back(1.0);
        }
    terms.push_back(identity_mpo(g.d()));
    coef.push_back(-2.0 * g.dims);
    return mpo_sum(coef, terms);
}

// Eq. 16 as one carry automaton with 2 dims + 1 bond states: D (nothing
// pending, identity from here on) and, per axis a, P_a / M_a (an increment /
// decrement along a still carrying).  The left boundary weighs D by -2 dims
// (-4 in 2D) and each shift state by 1 (every shift starts with its carry,
// Eq. 10); at a site of axis a, P_a keeps pending on bit 1 -> 0 and
// resolves to D on bit 0 -> 1, M_a the other way round; states of other
// axes pass by identity, D stays D.  The right boundary accepts every state
// (periodic) or only D (zero, Eq. 11).  Bond states that are zero on either
// side are removed, until no bond shrinks.  This is the gauge of the MPO the
// zip-up truncates in, which the step's result depends on.
Mpo laplacian_mpo(const Grid& g, int bc) {
    const int d = g.d(), ns = 2 * g.dims + 1, D = 0;
    std::vector<OpCore> W;
    for (int k = 0; k < d; ++k) {
        int axis, bit;
        site_axis(g, k, axis, bit);
        OpCore c(ns, ns);
        for (int s = 0; s < 2; ++s) c.at(D, s, s, D) = 1.0;
        for (int a = 0; a < g.dims; ++a) {
            const int p = 1 + 2 * a, m = 2 + 2 * a;
            if (a != axis) {
                for (int s = 0; s < 2; ++s) c.at(p, s, s, p) = c.at(m, s, s, m) = 1.0;
                continue;
            }
            c.at(p, 0, 1, p) = 1.0;  // increment: 1 -> 0, still carrying
            c.at(p, 1, 0, D) = 1.0;  // increment: 0 -> 1, done
            c.at(m, 1, 0, m) = 1.0;  // decrement: 0 -> 1, still borrowing
            c.at(m, 0, 1, D) = 1.0;  // decrement: 1 -> 0, done
        }
        W.push_back(c);
    }
    std::vector<double> inject(ns, 1.0);
    inject[D] = -2.0 * g.dims;
    OpCore first(1, ns);
    for (int a = 0; a < ns; ++a)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s)
                for (int b = 0; b < ns; ++b) first.at(0, t, s, b) += inject[a] * W[0].at(a, t, s, b);
    W[0] = first;
    OpCore lastc(W[d - 1].l, 1);
    for (int a = 0; a < W[d - 1].l; ++a)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s)
                for (int b = 0; b < ns; ++b)
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
//   psi^{k+1} = round(theta).  src: the source point, or null.
Mps mps_step(const Grid& g, const Mpo& L, const Mps& c2, double lambda2, const Mps& prev, const Mps& cur, double eps,
             int chi, const int* src, double amp) {
    const Mps phi = zipup_lr(L, cur, eps, chi);
    const Mps eta = zipup_rl(diagonal_mpo(c2), phi, eps, chi);
    std::vector<double> coef = {2.0, -1.0, lambda2};
    std::vector<const Mps*> terms = {&cur, &prev, &eta};
    Mps e;
    if (src) {
        e = product_state(g, src);
        coef.push_back(amp);
        terms.push_back(&e);
    }
    return tt_round(mps_sum(coef, terms), eps, chi);
}

// ---------------------------------------------------------------------------
// The transition operator of Eq. 7 as one MPO: A = 2I + lambda^2 C^2 L
// ---------------------------------------------------------------------------
// Operator product W_out W_in (W_in acts first): core k is
// sum_u W_out[a][t][u][a'] W_in[b][u][s][b'] on the bond pairs (a, b).
Mpo mpo_product(const Mpo& Wout, const Mpo& Win) {
    Mpo out;
    for (size_t k = 0; k < Wout.size(); ++k) {
        const OpCore &A = Wout[k], &B = Win[k];
        OpCore P(A.l * B.l, A.r * B.r);
        for (int a = 0; a < A.l; ++a)
            for (int b = 0; b < B.l; ++b)
                for (int t = 0; t < 2; ++t)
                    for (int s = 0; s < 2; ++s)
                        for (int a2 = 0; a2 < A.r; ++a2)
                            for (int b2 = 0; b2 < B.r; ++b2) {
                                double v = 0.0;
                                for (int u = 0; u < 2; ++u) v += A.at(a, t, u, a2) * B.at(b, u, s, b2);
                                P.at(a * B.l + b, t, s, a2 * B.r + b2) = v;
                            }
        out.push_back(P);
    }
    return out;
}

// A = 2I + lambda^2 C^2 L (Eq. 7): the diagonal MPO of c^2 times the
// Laplacian MPO, plus twice the identity (bond r_c w + 1).  The paper gives
// no representation; the reading shared with the library: the norm nu of the
// last c^2 core (which holds the whole norm of c^2 after TT-SVD) moves into
// the coefficient, lambda^2 nu, so that the two terms are of comparable size
// at every cut the zip-up makes.  The operator is unchanged.
Mpo a_operator_mpo(const Mpo& L, const Mps& c2, double lambda2) {
    Mps B = c2;
    double nu = 0.0;
    for (double x : B.back().a) nu += x * x;
    nu = std::sqrt(nu);
    if (nu > 0.0) {
        for (double& x : B.back().a) x /= nu;
    } else {
        nu = 1.0;
    }
    return mpo_sum({lambda2 * nu, 2.0}, {mpo_product(diagonal_mpo(B), L), identity_mpo((int)L.size())});
}

// The step of Eq. 7 with A applied as one operator: phi = A psi^k (zip-up,
// sites 1 -> d); theta = phi - psi^{k-1} [+ amp e_src]; psi^{k+1} =
// round(theta).  Exactly the step of mps_step; the truncation points differ.
Mps mps_step_fused(const Grid& g, const Mpo& A, const Mps& prev, const Mps& cur, double eps, int chi, const int* src,
                   double amp) {
    const Mps phi = zipup_lr(A, cur, eps, chi);
    std::vector<double> coef = {1.0, -1.0};
    std::vector<const Mps*> terms = {&phi, &prev};
    Mps e;
    if (src) {
        e = product_state(g, src);
        coef.push_back(amp);
        terms.push_back(&e);
    }
    return tt_round(mps_sum(coef, terms), eps, chi);
}

// Operator matrix of an MPO on the dense grid: out[p * P + q] = <p|W|q>,
// P = N^dims points, p and q dense indices.
void mpo_grid_operator(const Grid& g, const Mpo& W, double* out) {
    const int64_t P = g.points();
    int po[3], pi[3];
    for (int64_t p = 0; p < P; ++p) {
        coords(g, p, po);
        for (int64_t q = 0; q < P; ++q) {
            coords(g, q, pi);
            std::vector<double> v(1, 1.0);
            for (int k = 0; k < g.d(); ++k) {
                int axis, bit;
                site_axis(g, k, axis, bit);
                const int t = (po[axis] >> bit) & 1, s = (pi[axis] >> bit) & 1;
                std::vector<double> nv(W[k].r, 0.0);
                for (int a = 0; a < W[k].l; ++a)
                    for (int b = 0; b < W[k].r; ++b) nv[b] += v[a] * W[k].at(a, t, s, b);
                v.swap(nv);
            }
            out[p * P + q] = v[0];
        }
    }
}

// ---------------------------------------------------------------------------
// Dense FDTD (Sec. 2, Eq. 2; the 7-point stencil in 3D)
// ---------------------------------------------------------------------------
// u^{k+1} = 2 u^k - u^{k-1} + lambda^2 c^2 (sum of the 2 dims face
// neighbours - 2 dims u^k), neighbours by the boundary rule (periodic wrap
// or zero outside), plus amp at the source point (src may be null).
void fdtd_step(const Grid& g, const double* prev, const double* cur, const double* c2, double lambda2, int bc,
               const int* src, double amp, double* out) {
    const int N = g.N();
    int p[3], q[3];
    for (int64_t lin = 0; lin < g.points(); ++lin) {
        coords(g, lin, p);
        double nb = 0.0;
        for (int a = 0; a < g.dims; ++a)
            for (int step : {+1, -1}) {
                for (int b = 0; b < g.dims; ++b) q[b] = p[b];
                q[a] += step;
                if (bc == 0) {
                    q[a] = (q[a] + N) % N;
                } else if (q[a] < 0 || q[a] >= N) {
                    continue;
                }
                int64_t j = 0;
                for (int b = 0; b < g.dims; ++b) j = j * N + q[b];
                nb += cur[j];
            }
        out[lin] = 2.0 * cur[lin] - prev[lin] + lambda2 * c2[lin] * (nb - 2.0 * g.dims * cur[lin]);
    }
    if (src) {
        int64_t j = 0;
        for (int b = 0; b < g.dims; ++b) j = j * N + src[b];
        out[j] += amp;
    }
}

// ---------------------------------------------------------------------------
// Learned rank proposal and randomised rounding (the learned form)
// ---------------------------------------------------------------------------
// The paper rounds every bond with a full SVD (Sec. 4.3); the learned form
// keeps that rule as the arbiter.  A small MLP (40 features -> 128 -> 128 ->
// 1, ReLU) proposes a bond's rank for the next step from its spectrum; the
// round then first tries a randomised range finder of width r_hat + p
// (Halko, Martinsson & Tropp, SIAM Review 2011, Algorithm 4.1 and the direct
// SVD of Sec. 5.1) and keeps it only if an exact check says the Sec. 4.3 cut
// is inside the sketch; otherwise the bond takes the full SVD.
constexpr int kFeat = 40, kWidth = 128, kSpec = 32;
constexpr int kParams = kWidth * kFeat + kWidth + kWidth * kWidth + kWidth + kWidth + 1;

// The 40 features of a bond's spectrum S (L descending values) after a cut
// that kept r values, threshold eps, cap chi, bond k of d:
//   0..31 log10(S_p / S_0) at p = floor(j (L-1) / 31), clipped to [-16, 0],
//         over 16 (-1 when S_0 or S_p is 0); 32 r / chi; 33 log10 of the
//         discarded weight over S_0^2, clipped to [-32, 0], over 32 (-1 when
//         none); 34 log10(eps) / 16; 35 k / d; 36 min(2^k, 2^(d-k), chi) /
//         chi; 37 #{S_i >= eps S_0} / chi; 38 L / (2 chi); 39 one.
void rank_features(const double* S, int L, int r, double eps, int chi, int k, int d, double* f) {
    const double s0 = L > 0 ? S[0] : 0.0;
    for (int j = 0; j < kSpec; ++j) {
        const int p = L > 1 ? (j * (L - 1)) / (kSpec - 1) : 0;
        f[j] = (s0 > 0.0 && L > 0 && S[p] > 0.0) ? std::min(std::max(std::log10(S[p] / s0), -16.0), 0.0) / 16.0 : -1.0;
    }
    f[32] = (double)r / chi;
    double disc = 0.0;
    for (int i = r; i < L; ++i) disc += S[i] * S[i];
    f[33] = (s0 > 0.0 && disc > 0.0) ? std::min(std::max(std::log10(disc / (s0 * s0)), -32.0), 0.0) / 32.0 : -1.0;
    f[34] = eps > 0.0 ? std::log10(eps) / 16.0 : -1.0;
    f[35] = (double)k / d;
    f[36] = std::min({std::ldexp(1.0, k), std::ldexp(1.0, d - k), (double)chi}) / chi;
    int above = 0;
    if (s0 > 0.0)
        for (int i = 0; i < L; ++i) above += S[i] >= eps * s0;
    f[37] = (double)above / chi;
    f[38] = L / (2.0 * chi);
    f[39] = 1.0;
}

// Parameters, flat: W1 (128 x 40), b1, W2 (128 x 128), b2, W3 (1 x 128), b3.
struct MlpView {
    const double *W1, *b1, *W2, *b2, *W3, *b3;
    explicit MlpView(const double* p)
        : W1(p), b1(W1 + kWidth * kFeat), W2(b1 + kWidth), b2(W2 + kWidth * kWidth), W3(b2 + kWidth),
          b3(W3 + kWidth) {}
};

// y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each of the n rows x of X;
// the pre-activations a1, a2 (n x 128) are kept for the backward pass.
void mlp_forward(const double* p, const double* X, int n, double* y, std::vector<double>& a1,
                 std::vector<double>& a2) {
    const MlpView w(p);
    a1.assign((size_t)n * kWidth, 0.0);
    a2.assign((size_t)n * kWidth, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int u = 0; u < kWidth; ++u) {
            double acc = w.b1[u];
            for (int f = 0; f < kFeat; ++f) acc += w.W1[u * kFeat + f] * X[i * kFeat + f];
            a1[(size_t)i * kWidth + u] = acc;
        }
        for (int u = 0; u < kWidth; ++u) {
            double acc = w.b2[u];
            for (int v = 0; v < kWidth; ++v) acc += w.W2[u * kWidth + v] * std::max(a1[(size_t)i * kWidth + v], 0.0);
            a2[(size_t)i * kWidth + u] = acc;
        }
        double acc = w.b3[0];
        for (int v = 0; v < kWidth; ++v) acc += w.W3[v] * std::max(a2[(size_t)i * kWidth + v], 0.0);
        y[i] = acc;
    }
}

// Mean squared error of y against t and its gradient with respect to every
// parameter (chain rule through the three layers; ReLU' = [a > 0]).
double mlp_grad(const double* p, const double* X, const double* t, int n, double* g) {
    const MlpView w(p);
    std::vector<double> y(n), a1, a2;
    mlp_forward(p, X, n, y.data(), a1, a2);
    std::fill(g, g + kParams, 0.0);
    double* gW1 = g;
    double* gb1 = gW1 + kWidth * kFeat;
    double* gW2 = gb1 + kWidth;
    double* gb2 = gW2 + kWidth * kWidth;
    double* gW3 = gb2 + kWidth;
    double* gb3 = gW3 + kWidth;
    double loss = 0.0;
    std::vector<double> da2(kWidth), da1(kWidth);
    for (int i = 0; i < n; ++i) {
        const double e = y[i] - t[i];
        loss += e * e;
        const double dy = 2.0 * e / n;
        const double* A1 = &a1[(size_t)i * kWidth];
        const double* A2 = &a2[(size_t)i * kWidth];
        gb3[0] += dy;
        for (int v = 0; v < kWidth; ++v) {
            gW3[v] += dy * std::max(A2[v], 0.0);
            da2[v] = A2[v] > 0.0 ? dy * w.W3[v] : 0.0;
        }
        for (int u = 0; u < kWidth; ++u) {
            gb2[u] += da2[u];
            for (int v = 0; v < kWidth; ++v) gW2[u * kWidth + v] += da2[u] * std::max(A1[v], 0.0);
        }
        for (int v = 0; v < kWidth; ++v) {
            double acc = 0.0;
            for (int u = 0; u < kWidth; ++u) acc += da2[u] * w.W2[u * kWidth + v];
            da1[v] = A1[v] > 0.0 ? acc : 0.0;
        }
        for (int u = 0; u < kWidth; ++u) {
            gb1[u] += da1[u];
            for (int f = 0; f < kFeat; ++f) gW1[u * kFeat + f] += da1[u] * X[i * kFeat + f];
        }
    }
    return loss / n;
}

// One Adam update (Kingma & Ba, Algorithm 1), step t counted from 1.
void adam_step(double* p, const double* g, double* m, double* v, int np, int t, double lr, double beta1,
               double beta2, double eps) {
    for (int i = 0; i < np; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        const double mh = m[i] / (1.0 - std::pow(beta1, t)), vh = v[i] / (1.0 - std::pow(beta2, t));
        p[i] -= lr * mh / (std::sqrt(vh) + eps);
    }
}

// The range finder for the Sec. 4.3 cut of X (l x m) from a sketch of its
// row space with the Gaussian Omega (l x ks):
//   Y = X^T Omega, Q = qr(Y), B = Q^T X^T, B = Ub diag(Sb) Vb^T,
//   X ~ Vb diag(Sb) (Q Ub)^T, rho = ||X - X Q Q^T||_F (explicitly).
// With c = #{Sb_i >= eps Sb_0}: the sketch is rejected when c >= ks (the
// cut is not inside it); below the cap it is accepted iff rho <= eps Sb_0
// (every discarded direction of X is then below sqrt(2) eps sigma_1); at
// the cap iff rho^2 <= ((1 + tau)^2 - 1) sum_{i >= chi} Sb_i^2 (its
// discarded weight is then within (1 + tau)^2 of the optimum, by Ky Fan's
// principle on X X^T = A A^T + E E^T).  Outputs: r, Vt (r x m) and
// US (l x r) with X ~ US Vt, Sb, rho.
bool range_finder_svd(const Mat& X, const Mat& Om, double eps, int chi, double tau, int& r, Mat& Vt, Mat& US,
                      std::vector<double>& Sb, double& rho) {
    const int l = X.m, m = X.n, ks = Om.n;
    Mat Y(m, ks);  // X^T Omega
    for (int i = 0; i < l; ++i)
        for (int a = 0; a < m; ++a) {
            const double x = X(i, a);
            for (int j = 0; j < ks; ++j) Y(a, j) += x * Om(i, j);
        }
    Mat Q, R;
    householder_qr(Y, Q, R);
    const int q = Q.n;
    Mat XQ(l, q);  // X Q, so B = (X Q)^T
    for (int i = 0; i < l; ++i)
        for (int a = 0; a < m; ++a) {
            const double x = X(i, a);
            for (int j = 0; j < q; ++j) XQ(i, j) += x * Q(a, j);
        }
    const Mat B = transpose(XQ);  // q x l
    Mat Ub, Vbt;
    jacobi_svd(B, Ub, Sb, Vbt);
    double e2 = 0.0;
    for (int i = 0; i < l; ++i)
        for (int a = 0; a < m; ++a) {
            double proj = 0.0;
            for (int j = 0; j < q; ++j) proj += XQ(i, j) * Q(a, j);
            const double e = X(i, a) - proj;
            e2 += e * e;
        }
    rho = std::sqrt(e2);
    const double s0 = Sb.empty() ? 0.0 : Sb[0];
    int c = 0;
    if (s0 > 0.0)
        for (double s : Sb) c += s >= eps * s0;
    r = trunc_rank(Sb, eps, chi);
    bool ok;
    if (s0 == 0.0) {
        ok = rho == 0.0;
    } else if (c >= ks) {
        ok = false;
    } else if (c < chi) {
        ok = rho <= eps * s0;
    } else {
        double tail = 0.0;
        for (size_t i = chi; i < Sb.size(); ++i) tail += Sb[i] * Sb[i];
        ok = rho * rho <= ((1.0 + tau) * (1.0 + tau) - 1.0) * tail;
    }
    Vt = Mat(r, m);  // (Q Ub[:, :r])^T
    for (int j = 0; j < r; ++j)
        for (int a = 0; a < m; ++a) {
            double acc = 0.0;
            for (int b = 0; b < q; ++b) acc += Q(a, b) * Ub(b, j);
            Vt(j, a) = acc;
        }
    US = Mat(l, r);  // Vb[:, :r] diag(Sb[:r])
    for (int i = 0; i < l; ++i)
        for (int j = 0; j < r; ++j) US(i, j) = Vbt(j, i) * Sb[j];
    return ok;
}

// The round of Sec. 4.3 where bond k of the SVD sweep first tries the range
// finder of width ks = proposals[k] + p, with Omega the top-left l x ks block
// of one fixed Gaussian matrix G, when ks < min(l, 2 r_k); rejected or
// unproposed bonds take the full SVD.  log receives (k, ks, accepted).
// A G smaller than l x ks makes the bond unproposed.
Mps tt_round_learned(Mps A, double eps, int chi, const int* proposals, const Mat& G, int p, double tau,
                     std::vector<int>* log) {
    const int d = (int)A.size();
    for (int k = 0; k + 1 < d; ++k) {
        Mat M(A[k].l * 2, A[k].r);
        M.a = A[k].a;
        Mat Q, R;
        householder_qr(M, Q, R);
        const int kk = Q.n;
        Core qc(A[k].l, kk);
        qc.a = Q.a;
        const Core& nx = A[k + 1];
        Core nn(kk, nx.r);
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < nx.l; ++j)
                for (int s = 0; s < 2; ++s)
                    for (int e = 0; e < nx.r; ++e) nn.at(i, s, e) += R(i, j) * nx.at(j, s, e);
        A[k] = std::move(qc);
        A[k + 1] = std::move(nn);
    }
    for (int k = d - 1; k > 0; --k) {
        const int l = A[k].l, rr2 = 2 * A[k].r;
        Mat X(l, rr2);
        X.a = A[k].a;
        int r = 0;
        Mat Vt, US;
        bool done = false;
        const int ph = proposals ? proposals[k] : 0;
        // (a G too small for this bond counts as no proposal)
        if (ph > 0 && ph + p < std::min(l, rr2) && l <= G.m && ph + p <= G.n) {
            const int ks = ph + p;
            Mat Om(l, ks);
            for (int i = 0; i < l; ++i)
                for (int j = 0; j < ks; ++j) Om(i, j) = G(i, j);
            std::vector<double> Sb;
            double rho;
            const bool ok = range_finder_svd(X, Om, eps, chi, tau, r, Vt, US, Sb, rho);
            if (log) log->insert(log->end(), {k, ks, ok ? 1 : 0});
            done = ok;
        }
        if (!done) {
            Mat U, V;
            std::vector<double> S;
            jacobi_svd(X, U, S, V);
            r = trunc_rank(S, eps, chi);
            Vt = Mat(r, rr2);
            for (int i = 0; i < r; ++i)
                for (int j = 0; j < rr2; ++j) Vt(i, j) = V(i, j);
            US = Mat(l, r);
            for (int i = 0; i < l; ++i)
                for (int j = 0; j < r; ++j) US(i, j) = U(i, j) * S[j];
        }
        Core v(r, A[k].r);
        v.a = Vt.a;
        const Core& pv = A[k - 1];
        Core np(pv.l, r);
        for (int a = 0; a < pv.l; ++a)
            for (int s = 0; s < 2; ++s)
                for (int j = 0; j < pv.r; ++j)
                    for (int e = 0; e < r; ++e) np.at(a, s, e) += pv.at(a, s, j) * US(j, e);
        A[k] = std::move(v);
        A[k - 1] = std::move(np);
    }
    return A;
}

Mps* box(Mps&& m) { return new Mps(std::move(m)); }
Mpo* box(Mpo&& m) { return new Mpo(std::move(m)); }
}  // namespace

// ---------------------------------------------------------------------------
// C interface for the tests (ctypes).  Handles own their cores; every call
// that returns a handle returns a new one.  No call throws or exits.
// ---------------------------------------------------------------------------
extern "C" {

// Grids are passed as (dims, n, order): dims 2 or 3, order 0 = SEQUENTIAL,
// 1 = INTERLEAVED; boundaries as bc 0 = PERIODIC, 1 = ZERO; points as dims
// ints; dense fields as N^dims doubles in the layout of the Grid comment.

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

void* oc_mps_from_dense(int dims, int n, int order, const double* u, double eps, int chi) {
    return box(mps_from_dense(Grid{dims, n, order}, u, eps, chi));
}
void oc_mps_to_dense(const void* h, int dims, int n, int order, double* u) {
    mps_to_dense(Grid{dims, n, order}, *static_cast<const Mps*>(h), u);
}
void oc_mps_sample(const void* h, int dims, int n, int order, int np, const int* pts, double* out) {
    for (int p = 0; p < np; ++p) out[p] = mps_sample(Grid{dims, n, order}, *static_cast<const Mps*>(h), pts + p * dims);
}
void* oc_product_state(int dims, int n, int order, const int* p) {
    return box(product_state(Grid{dims, n, order}, p));
}
void* oc_round(const void* h, double eps, int chi) { return box(tt_round(*static_cast<const Mps*>(h), eps, chi)); }
void* oc_sum(int nterms, const double* coef, void* const* terms) {
    std::vector<double> c(coef, coef + nterms);
    std::vector<const Mps*> t;
    for (int j = 0; j < nterms; ++j) t.push_back(static_cast<const Mps*>(terms[j]));
    return box(mps_sum(c, t));
}

void* oc_shift_mpo(int dims, int n, int order, int axis, int sign, int bc) {
    return box(shift_mpo(Grid{dims, n, order}, axis, sign, bc));
}
void* oc_laplacian_mpo(int dims, int n, int order, int bc) { return box(laplacian_mpo(Grid{dims, n, order}, bc)); }
void* oc_laplacian_sum_of_shifts(int dims, int n, int order, int bc) {
    return box(laplacian_sum_of_shifts(Grid{dims, n, order}, bc));
}
void* oc_diagonal_mpo(const void* h) { return box(diagonal_mpo(*static_cast<const Mps*>(h))); }
void* oc_a_operator_mpo(const void* L, const void* c2, double lambda2) {
    return box(a_operator_mpo(*static_cast<const Mpo*>(L), *static_cast<const Mps*>(c2), lambda2));
}
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
void oc_mpo_grid_operator(const void* h, int dims, int n, int order, double* out) {
    mpo_grid_operator(Grid{dims, n, order}, *static_cast<const Mpo*>(h), out);
}
void oc_mpo_free(void* h) { delete static_cast<Mpo*>(h); }

void* oc_zipup_lr(const void* W, const void* A, double eps, int chi) {
    return box(zipup_lr(*static_cast<const Mpo*>(W), *static_cast<const Mps*>(A), eps, chi));
}
void* oc_zipup_rl(const void* W, const void* A, double eps, int chi) {
    return box(zipup_rl(*static_cast<const Mpo*>(W), *static_cast<const Mps*>(A), eps, chi));
}
void* oc_step(const void* L, const void* c2, double lambda2, const void* prev, const void* cur, double eps, int chi,
              const int* src, double amp, int dims, int n, int order) {
    return box(mps_step(Grid{dims, n, order}, *static_cast<const Mpo*>(L), *static_cast<const Mps*>(c2), lambda2,
                        *static_cast<const Mps*>(prev), *static_cast<const Mps*>(cur), eps, chi, src, amp));
}
void* oc_step_fused(const void* A, const void* prev, const void* cur, double eps, int chi, const int* src, double amp,
                    int dims, int n, int order) {
    return box(mps_step_fused(Grid{dims, n, order}, *static_cast<const Mpo*>(A), *static_cast<const Mps*>(prev),
                              *static_cast<const Mps*>(cur), eps, chi, src, amp));
}
void oc_fdtd_step(int dims, int n, const double* prev, const double* cur, const double* c2, double lambda2, int bc,
                  const int* src, double amp, double* out) {
    fdtd_step(Grid{dims, n, 0}, prev, cur, c2, lambda2, bc, src, amp, out);
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

// ---- learned form ----
int oc_mlp_param_count(void) { return kParams; }
void oc_rank_features(const double* S, int L, int r, double eps, int chi, int k, int d, double* f) {
    rank_features(S, L, r, eps, chi, k, d, f);
}
void oc_mlp_forward(const double* p, const double* X, int n, double* y) {
    std::vector<double> a1, a2;
    mlp_forward(p, X, n, y, a1, a2);
}
double oc_mlp_grad(const double* p, const double* X, const double* t, int n, double* g) {
    return mlp_grad(p, X, t, n, g);
}
void oc_adam_step(double* p, const double* g, double* m, double* v, int np, int t, double lr, double beta1,
                  double beta2, double eps) {
    adam_step(p, g, m, v, np, t, lr, beta1, beta2, eps);
}
// Returns accepted (0/1); writes r, Vt (r x m, room for min(l, ks) x m),
// US (l x r, room for l x min(l, ks)), Sb (room for min(l, ks)) and rho.
int oc_range_finder_svd(int l, int m, const double* X, int ks, const double* Om, double eps, int chi, double tau,
                        int* r_out, double* Vt, double* US, double* Sb, int* nsb, double* rho) {
    Mat x(l, m), om(l, ks);
    std::memcpy(x.a.data(), X, x.a.size() * sizeof(double));
    std::memcpy(om.a.data(), Om, om.a.size() * sizeof(double));
    int r;
    Mat vt, us;
    std::vector<double> sb;
    const bool ok = range_finder_svd(x, om, eps, chi, tau, r, vt, us, sb, *rho);
    *r_out = r;
    *nsb = (int)sb.size();
    std::memcpy(Vt, vt.a.data(), vt.a.size() * sizeof(double));
    std::memcpy(US, us.a.data(), us.a.size() * sizeof(double));
    std::memcpy(Sb, sb.data(), sb.size() * sizeof(double));
    return ok ? 1 : 0;
}
// proposals: d ints or null; G (gl x gk) row-major; log: room for 3 (d - 1)
// ints, *nlog receives the count of ints written.
void* oc_round_learned(const void* h, double eps, int chi, const int* proposals, int gl, int gk, const double* G,
                       int p, double tau, int* log, int* nlog) {
    Mat g(gl, gk);
    std::memcpy(g.a.data(), G, g.a.size() * sizeof(double));
    std::vector<int> lg;
    Mps out = tt_round_learned(*static_cast<const Mps*>(h), eps, chi, proposals, g, p, tau, &lg);
    std::copy(lg.begin(), lg.end(), log);
    *nlog = (int)lg.size();
    return box(std::move(out));
}

int oc_trunc_rank(int p, const double* s, double eps, int chi) {
    return trunc_rank(std::vector<double>(s, s + p), eps, chi);
}

}  // extern "C"
