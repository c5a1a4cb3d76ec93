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
#include <vector>

#include "qtt_internal.cuh"

namespace qtt {

namespace {
enum { SD = 0, SXP = 1, SXM = 2, SZP = 3, SZM = 4, NS = 5 };

inline double& at(std::vector<double>& w, int l, int t, int s, int r) { return w[((l * 2 + t) * 2 + s) * NS + r]; }

void put(std::vector<double>& w, int l, int r, int op) {
  // op: 0 = I, 1 = sigma^+ = |1><0|, 2 = sigma^- = |0><1|; entries [t][s]
  if (op == 0) {
    at(w, l, 0, 0, r) = 1.0;
    at(w, l, 1, 1, r) = 1.0;
  } else if (op == 1) {
    at(w, l, 1, 0, r) = 1.0;
  } else {
    at(w, l, 0, 1, r) = 1.0;
  }
}
}  // namespace

// Fills mpo->w, mpo->off, mpo->host.
void build_laplacian(int n, int order, int bc, Mpo* mpo) {
  const int d = 2 * n;
  // full 5-state cores, [l][t][s][r]
  std::vector<std::vector<double>> W(d, std::vector<double>(NS * 4 * NS, 0.0));
  for (int k = 0; k < d; ++k) {
    const bool is_x = (order == QTT_ORDER_SEQUENTIAL) ? (k < n) : ((k & 1) == 0);
    const int p = is_x ? SXP : SZP, m = is_x ? SXM : SZM;
    const int op = is_x ? SZP : SXP, om = is_x ? SZM : SXM;
    put(W[k], SD, SD, 0);
    put(W[k], p, p, 2);
    put(W[k], p, SD, 1);
    put(W[k], m, m, 1);
    put(W[k], m, SD, 2);
    put(W[k], op, op, 0);
    put(W[k], om, om, 0);
  }
  const double inject[NS] = {-4.0, 1.0, 1.0, 1.0, 1.0};
  double accept[NS] = {1.0, 1.0, 1.0, 1.0, 1.0};
  if (bc == QTT_BC_ZERO) accept[1] = accept[2] = accept[3] = accept[4] = 0.0;

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
              if (at(W[k - 1], l, t, u, s) != 0.0) { in = true; break; }
        }
        for (int r = 0; r < NS && !out; ++r) {
          bool rr = (k + 1 == d) ? rb[r] : live[k + 1][r];
          if (!rr) continue;
          for (int t = 0; t < 2 && !out; ++t)
            for (int u = 0; u < 2; ++u)
              if (at(W[k], s, t, u, r) != 0.0) { out = true; break; }
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
                v += wlv * at(W[k], l, t, u, r) * wrv;
              }
            }
            dst[((li * 2 + t) * 2 + u) * wr + ri] = v;
          }
  }
}

}  // namespace qtt
