// Host builder of the Laplacian MPO (Eq. 16) from the carry tensors of the
// shift operators (Eq. 9-13), for both site orders and both boundary rules.
//
// Sites run least significant bit first (the tensor-product order of
// Eq. 12).  One automaton with five bond states carries the whole sum
// S_x^+ + S_x^- + S_z^+ + S_z^- - 4I:
//   D   no carry pending (identity on the remaining sites),
//   XP  S_x^+ with a carry pending,   XM  S_x^- with a borrow pending,
//   ZP  S_z^+ with a carry pending,   ZM  S_z^- with a borrow pending.
// The left boundary injects -4 on D and 1 on each shift state (the carry 1
// of Eq. 10); an x site maps XP->XP by sigma^- and XP->D by sigma^+ (the
// two entries of the second row of Eq. 9), XM->XM by sigma^+ and XM->D by
// sigma^- (Eq. 13), passes the z states through and keeps D by I.  The
// right boundary accepts every state for the periodic shift (the overflow
// wraps, Sec. 3.1) or only D for the zero-outside shift (Eq. 11 as
// printed).  Bond states that vanish on either side are dropped.
//
// The 3D extension (the paper's discussion section) adds the pair of y
// shifts: seven bond states (D, then S^+ and S^- per axis), -6 injected on D
// (the 7-point stencil), each site acting on the states of its own axis and
// passing the others through.
#include <cmath>
#include <vector>

#include "qtt_internal.cuh"

namespace qtt {

namespace {
// bond states: 0 = D (no carry pending), 1 + 2a / 2 + 2a = S_a^+ / S_a^- of
// axis a with a carry / borrow pending (2D: D, XP, XM, ZP, ZM)
constexpr int kMaxStates = 7;
constexpr int SD = 0;

inline double& at(std::vector<double>& w, int ns, int l, int t, int s, int r) {
  return w[((l * 2 + t) * 2 + s) * ns + r];
}

void put(std::vector<double>& w, int ns, int l, int r, int op) {
  // op: 0 = I, 1 = sigma^+ = |1><0|, 2 = sigma^- = |0><1|; entries [t][s]
  if (op == 0) {
    at(w, ns, l, 0, 0, r) = 1.0;
    at(w, ns, l, 1, 1, r) = 1.0;
  } else if (op == 1) {
    at(w, ns, l, 1, 0, r) = 1.0;
  } else {
    at(w, ns, l, 0, 1, r) = 1.0;
  }
}
}  // namespace

// Axis of site k: SEQUENTIAL puts the registers one after another (Eq. 14-15),
// INTERLEAVED cycles through the axes; the least significant bit comes first.
int site_axis(int k, int n, int order, int dims) { return order == QTT_ORDER_SEQUENTIAL ? k / n : k % dims; }

// Bit of the linear dense index ((x N + y) N + z, or x N + z in 2D) that
// site k carries.
int site_pos(int k, int n, int order, int dims) {
  const int axis = site_axis(k, n, order, dims);
  const int bit = order == QTT_ORDER_SEQUENTIAL ? k % n : k / dims;
  return n * (dims - 1 - axis) + bit;
}

// Fills mpo->w, mpo->off, mpo->host: the 5-point (2D) or 7-point (3D)
// Laplacian sum_a (S_a^+ + S_a^-) - 2 dims I.
void build_laplacian(int n, int order, int bc, int dims, Mpo* mpo) {
  const int d = dims * n, NS = 2 * dims + 1;
  // full cores, [l][t][s][r]
  std::vector<std::vector<double>> W(d, std::vector<double>(NS * 4 * NS, 0.0));
  for (int k = 0; k < d; ++k) {
    const int a = site_axis(k, n, order, dims);
    put(W[k], NS, SD, SD, 0);
    for (int b = 0; b < dims; ++b) {
      const int p = 1 + 2 * b, m = 2 + 2 * b;
      if (b == a) {
        put(W[k], NS, p, p, 2);
        put(W[k], NS, p, SD, 1);
        put(W[k], NS, m, m, 1);
        put(W[k], NS, m, SD, 2);
      } else {
        put(W[k], NS, p, p, 0);
        put(W[k], NS, m, m, 0);
      }
    }
  }
  double inject[kMaxStates], accept[kMaxStates];
  for (int s = 0; s < NS; ++s) {
    inject[s] = s == SD ? -2.0 * dims : 1.0;
    accept[s] = (s == SD || bc != QTT_BC_ZERO) ? 1.0 : 0.0;
  }

  // live states per bond: nonzero on both sides (after folding the boundaries)
  std::vector<std::vector<int>> keep(d + 1);
  keep[0] = {0};
  keep[d] = {0};
  std::vector<std::vector<char>> live(d + 1, std::vector<char>(NS, 1));
  // iterate to a fixed point: state s at bond k (1..d-1) is live if W[k-1]
  // has a nonzero entry into it from a live left state and W[k] has one out
  // of it into a live right state
  std::vector<char> lb(NS), rb(NS);
  for (int s = 0; s < NS; ++s) {
    lb[s] = inject[s] != 0.0;
    rb[s] = accept[s] != 0.0;
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int k = 1; k < d; ++k) {
      for (int s = 0; s < NS; ++s) {
        if (!live[k][s]) continue;
        bool in = false, out = false;
        for (int l = 0; l < NS && !in; ++l) {
          bool ll = (k - 1 == 0) ? lb[l] : live[k - 1][l];
          if (!ll) continue;
          for (int t = 0; t < 2 && !in; ++t)
            for (int u = 0; u < 2; ++u)
              if (at(W[k - 1], NS, l, t, u, s) != 0.0) { in = true; break; }
        }
        for (int r = 0; r < NS && !out; ++r) {
          bool rr = (k + 1 == d) ? rb[r] : live[k + 1][r];
          if (!rr) continue;
          for (int t = 0; t < 2 && !out; ++t)
            for (int u = 0; u < 2; ++u)
              if (at(W[k], NS, s, t, u, r) != 0.0) { out = true; break; }
        }
        if (!(in && out)) {
          live[k][s] = 0;
          changed = true;
        }
      }
    }
  }
  for (int k = 1; k < d; ++k)
    for (int s = 0; s < NS; ++s)
      if (live[k][s]) keep[k].push_back(s);

  mpo->d = d;
  mpo->w.assign(d + 1, 1);
  mpo->off.assign(d, 0);
  for (int k = 1; k < d; ++k) mpo->w[k] = (int)keep[k].size();
  long long tot = 0;
  for (int k = 0; k < d; ++k) {
    mpo->off[k] = tot;
    tot += (long long)mpo->w[k] * 4 * mpo->w[k + 1];
  }
  mpo->host.assign(tot, 0.0);
  for (int k = 0; k < d; ++k) {
    const int wl = mpo->w[k], wr = mpo->w[k + 1];
    double* dst = mpo->host.data() + mpo->off[k];
    for (int li = 0; li < wl; ++li)
      for (int t = 0; t < 2; ++t)
        for (int u = 0; u < 2; ++u)
          for (int ri = 0; ri < wr; ++ri) {
            double v = 0.0;
            // left side: boundary vector at k == 0, else the kept state
            for (int l = 0; l < NS; ++l) {
              double wlv = (k == 0) ? inject[l] : (l == keep[k][li] ? 1.0 : 0.0);
              if (wlv == 0.0) continue;
              for (int r = 0; r < NS; ++r) {
                double wrv = (k == d - 1) ? accept[r] : (r == keep[k + 1][ri] ? 1.0 : 0.0);
                if (wrv == 0.0) continue;
                v += wlv * at(W[k], NS, l, t, u, r) * wrv;
              }
            }
            dst[((li * 2 + t) * 2 + u) * wr + ri] = v;
          }
  }
}

}  // namespace qtt

namespace qtt {

// MPO of the transition operator of Eq. 7, A = 2I + lambda^2 C^2 L, on the
// host.  c2 holds the cores [r_k][2][r_{k+1}] of the c^2 MPS (ranks rc), L
// the Laplacian MPO.  The product C^2 L has cores B_k[r][t][r'] L_k[w][t][s][w']
// on the bond pair (r, w) (the diagonal MPO of c^2 acts on the output
// index); the sum with 2I appends one bond state carrying the identity.  The
// c^2 MPS keeps its norm (~c_max^2) in its last core: that norm nu is moved
// into the coefficient of the product term on the first core (lambda^2 nu),
// so that both terms are of order one at every bond the zip-up cuts; the
// operator is unchanged.
void build_a_operator(const Mpo& L, const std::vector<std::vector<double>>& c2, const std::vector<int>& rc,
                      double lambda2, Mpo* A) {
  const int d = L.d;
  double nu = 0.0;
  for (double v : c2[d - 1]) nu += v * v;
  nu = nu > 0.0 ? std::sqrt(nu) : 1.0;
  A->d = d;
  A->w.assign(d + 1, 1);
  for (int k = 1; k < d; ++k) A->w[k] = rc[k] * L.w[k] + 1;
  A->off.assign(d, 0);
  long long tot = 0;
  for (int k = 0; k < d; ++k) {
    A->off[k] = tot;
    tot += (long long)A->w[k] * 4 * A->w[k + 1];
  }
  A->host.assign(tot, 0.0);
  for (int k = 0; k < d; ++k) {
    const int wl = L.w[k], wr = L.w[k + 1], r0 = rc[k], r1 = rc[k + 1];
    const int Al = A->w[k], Ar = A->w[k + 1];
    const double* Lk = L.host.data() + L.off[k];
    const double* Bk = c2[k].data();
    const double coef = (k == 0) ? lambda2 * nu : 1.0;
    const double bscale = (k == d - 1) ? 1.0 / nu : 1.0;
    double* dst = A->host.data() + A->off[k];
    auto el = [&](int l, int t, int s, int r) -> double& { return dst[((l * 2 + t) * 2 + s) * Ar + r]; };
    // product block: left index r * wl + w (or 0 at k = 0), right r' * wr + w' (or 0 at the end)
    for (int r = 0; r < r0; ++r)
      for (int w = 0; w < wl; ++w)
        for (int t = 0; t < 2; ++t)
          for (int rp = 0; rp < r1; ++rp) {
            const double b = Bk[(r * 2 + t) * r1 + rp] * coef * bscale;
            if (b == 0.0) continue;
            for (int s = 0; s < 2; ++s)
              for (int wp = 0; wp < wr; ++wp) {
                const double l = Lk[((w * 2 + t) * 2 + s) * wr + wp];
                if (l == 0.0) continue;
                const int li = (k == 0) ? 0 : r * wl + w;
                const int ri = (k == d - 1) ? 0 : rp * wr + wp;
                el(li, t, s, ri) += b * l;
              }
          }
    // identity block: the last bond state, 2 delta_ts on the first core
    const int li = (k == 0) ? 0 : Al - 1;
    const int ri = (k == d - 1) ? 0 : Ar - 1;
    const double id = (k == 0) ? 2.0 : 1.0;
    el(li, 0, 0, ri) += id;
    el(li, 1, 1, ri) += id;
  }
}

}  // namespace qtt
