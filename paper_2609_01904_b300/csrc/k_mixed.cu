// Mixed-precision SVD of a small square bond factor (the reduced-precision
// form of the step).
//
// Stage 0, the preconditioning factor (Drmac & Veselic 2008): a graded
// triangular R whose rows are the Jacobi vectors, from a Cholesky with
// diagonal pivoting of the FP64 Gram matrix (pchol_cluster_kernel) or from a
// Householder QR with column pivoting of the small R0^T of a QR of the bond
// matrix (qrcp_cluster_kernel), each inside one thread-block cluster.
//
// Stage 1, FP32: one-sided Jacobi on the nv column vectors, all of them held
// in the shared memory of one thread-block cluster (columns split across the
// CTAs, partners reached through distributed shared memory), one hardware
// cluster barrier per round of the circle schedule.  It stops at 1e-4
// relative orthogonality, an order of magnitude above FP32 rounding.
//
// Stage 2, FP64 (host-driven GEMMs over the whole GPU, qtt_api.cu): Newton-
// Schulz re-orthonormalisation J <- J (3I - J^T J)/2, W = R J, G = W^T W, a
// simultaneous first-order Jacobi correction J <- J (I + Omega) with
// Omega_ij = G_ij / (G_jj - G_ii) (damped inside clusters of near-equal
// values), twice, then sigma_i = |W e_i| in FP64.  The rotation is
// orthogonal to FP64 rounding; the contamination of every vector by the
// directions of much larger values (FP32 rounding of the first stage) is
// removed, so well separated values come out to FP64 accuracy, while values
// within ~1e-7 sigma_1 of each other near the FP32 floor stay resolved only
// to about 1e-7 sigma_1.
#include <cooperative_groups.h>

#include <algorithm>

#include "k_mps.cuh"
#include "qtt_internal.cuh"

namespace cg = cooperative_groups;

namespace qtt {

namespace {

constexpr int NT32 = 512;

// One warp per pair.  Columns are zero-padded to multiples of 128 floats (a
// rotation keeps the padding zero), so a lane moves whole float4s: EA float4 of
// each vector and EJ of each rotation column per lane.  Column c lives in the
// shared memory of CTA c / cpc; its (distributed) address is looked up in a
// table built once, so a round is one batch of vector loads, three warp
// reductions, one batch of stores and one cluster barrier.
template <int EA, int EJ>
__global__ void __launch_bounds__(NT32) jacobi32_cluster_kernel(const double* __restrict__ V, long long ldv, Dim nv_d,
                                                                Dim m_d, double* __restrict__ Jout, long long ldj,
                                                                int cpc, int max_sweeps, float tol, float tol_abs,
                                                                int* log) {
  constexpr int MST = 128 * EA, JST = 128 * EJ;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CS = (int)cl.num_blocks();
  extern __shared__ float4 sm4[];
  float* A = reinterpret_cast<float*>(sm4);   // cpc columns of MST floats
  float* Jl = A + (long long)cpc * MST;       // cpc columns of JST floats
  float4** pa = reinterpret_cast<float4**>(Jl + (long long)cpc * JST);  // per-column addresses
  float4** pj = pa + (long long)cpc * CS;
  __shared__ int s_cnt;
  const int nv = (int)dv(nv_d), m = (int)dv(m_d);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT32 >> 5;

  for (int cl_i = 0; cl_i < cpc; ++cl_i) {
    const int c = rank * cpc + cl_i;
    for (int l = tid; l < MST; l += NT32) A[cl_i * MST + l] = (c < nv && l < m) ? (float)V[c * ldv + l] : 0.f;
    for (int l = tid; l < JST; l += NT32) Jl[cl_i * JST + l] = (c < nv && l == c) ? 1.f : 0.f;
  }
  for (int c = tid; c < cpc * CS; c += NT32) {
    pa[c] = reinterpret_cast<float4*>(cl.map_shared_rank(A + (c % cpc) * MST, c / cpc));
    pj[c] = reinterpret_cast<float4*>(cl.map_shared_rank(Jl + (c % cpc) * JST, c / cpc));
  }
  const int P = nv + (nv & 1), R = P - 1;
  int sweep = 0;
  for (sweep = 0; sweep < max_sweeps && nv >= 2; ++sweep) {
    if (tid == 0) s_cnt = 0;
    cl.sync();
    for (int rd = 0; rd < R; ++rd) {
      for (int q = rank + CS * warp; q < P / 2; q += CS * nw) {
        int i, j;
        if (q == 0) {
          i = R;
          j = rd;
        } else {
          i = rd + q;
          if (i >= R) i -= R;
          j = rd - q;
          if (j < 0) j += R;
        }
        if (i >= nv || j >= nv) continue;
        float4* xi = pa[i];
        float4* xj = pa[j];
        float4* ji = pj[i];
        float4* jj = pj[j];
        float4 x[EA], y[EA], u[EJ], w[EJ];
#pragma unroll
        for (int e = 0; e < EA; ++e) {
          x[e] = xi[lane + 32 * e];
          y[e] = xj[lane + 32 * e];
        }
#pragma unroll
        for (int e = 0; e < EJ; ++e) {
          u[e] = ji[lane + 32 * e];
          w[e] = jj[lane + 32 * e];
        }
        float a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
        for (int e = 0; e < EA; ++e) {
          a = fmaf(x[e].x, x[e].x, fmaf(x[e].y, x[e].y, fmaf(x[e].z, x[e].z, fmaf(x[e].w, x[e].w, a))));
          b = fmaf(y[e].x, y[e].x, fmaf(y[e].y, y[e].y, fmaf(y[e].z, y[e].z, fmaf(y[e].w, y[e].w, b))));
          g = fmaf(x[e].x, y[e].x, fmaf(x[e].y, y[e].y, fmaf(x[e].z, y[e].z, fmaf(x[e].w, y[e].w, g))));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (g != 0.f && fabsf(g) > tol * sqrtf(a) * sqrtf(b) && fabsf(g) > tol_abs * fmaxf(a, b)) {
          const float zeta = (b - a) / (2.f * g);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t), sn = cs * t;
#pragma unroll
          for (int e = 0; e < EA; ++e) {
            const float4 p = x[e], r = y[e];
            xi[lane + 32 * e] = make_float4(cs * p.x - sn * r.x, cs * p.y - sn * r.y, cs * p.z - sn * r.z,
                                            cs * p.w - sn * r.w);
            xj[lane + 32 * e] = make_float4(sn * p.x + cs * r.x, sn * p.y + cs * r.y, sn * p.z + cs * r.z,
                                            sn * p.w + cs * r.w);
          }
#pragma unroll
          for (int e = 0; e < EJ; ++e) {
            const float4 p = u[e], r = w[e];
            ji[lane + 32 * e] = make_float4(cs * p.x - sn * r.x, cs * p.y - sn * r.y, cs * p.z - sn * r.z,
                                            cs * p.w - sn * r.w);
            jj[lane + 32 * e] = make_float4(sn * p.x + cs * r.x, sn * p.y + cs * r.y, sn * p.z + cs * r.z,
                                            sn * p.w + cs * r.w);
          }
          if (lane == 0) atomicAdd(&s_cnt, 1);
        }
      }
      cl.sync();
    }
    // rotations of this sweep over the cluster
    int total = 0;
    for (int r = 0; r < CS; ++r) total += *cl.map_shared_rank(&s_cnt, r);
    cl.sync();  // every CTA has read the counters before the next sweep resets them
    if (total == 0) break;
  }
  if (log && rank == 0 && tid == 0) {
    log[0] = nv;
    log[1] = m;
    log[2] = sweep + 1;
  }
  for (int cl_i = 0; cl_i < cpc; ++cl_i) {
    const int c = rank * cpc + cl_i;
    if (c >= nv) continue;
    for (int l = tid; l < nv; l += NT32) Jout[(long long)c * ldj + l] = (double)Jl[cl_i * JST + l];
  }
}

// Block one-sided Jacobi with the Gram matrix of each block pair (the block
// method of Becka, Oksa & Vajtersic: a block pair is orthogonalised by the
// eigenvectors of its 2B x 2B Gram matrix, applied to the pair as one small
// product).  The nv columns form 2*CS blocks of B columns, and a sweep is a
// round-robin tournament of the blocks (circle method, 2*CS - 1 block
// rounds); in each block round a CTA
//   1. pulls its two blocks (B columns each, rows of 2B floats in a working
//      area, vectors and rotation columns) from the CTAs that held them in the
//      previous block round, into the other of its two working areas,
//   2. forms their Gram matrix G = X^T X (FP32, every entry a plain dot
//      product, so its error is relative to |x_i| |x_j|),
//   3. runs the rotations of the block round on G two-sidedly, one phase and
//      one barrier per round of disjoint pairs: every entry of R^T G R comes
//      from four entries of G (double-buffered), the rotations are
//      accumulated in a 2B x 2B orthogonal V, and sixteen lanes compute the
//      next round's rotations from the same four-entry formula meanwhile.  The
//      rotation of a pair is the one one-sided Jacobi takes from the same
//      columns, and the two-sided updates keep every entry's error relative to
//      its own scale (Demmel & Veselic, the accuracy of Jacobi on positive
//      definite matrices),
//   4. if anything rotated, applies X <- X V and J <- J V as dense products
//      (one warp per row, V's column in registers).
// A rotation then costs a few shared-memory words of G instead of two vectors
// of length m, and the vector work becomes two dense 2B-wide products per
// block round, skipped where nothing rotates.
namespace jg {

// position (CTA, half) of block b in block round t of the circle method
__device__ __forceinline__ void owner(int b, int t, int NB, int CS, int& r, int& h) {
  if (b == NB - 1) {
    r = 0;
    h = 0;
  } else if (b == t) {
    r = 0;
    h = 1;
  } else {
    int d = b - t;
    if (d < 0) d += NB - 1;
    if (d >= 1 && d <= CS - 1) {
      r = d;
      h = 0;
    } else {
      d = t - b;
      if (d < 0) d += NB - 1;
      r = d;
      h = 1;
    }
  }
}

// the two blocks of CTA `rank` in block round t
__device__ __forceinline__ void blocks(int t, int rank, int NB, int& bp, int& bq) {
  if (rank == 0) {
    bp = NB - 1;
    bq = t;
  } else {
    bp = t + rank;
    if (bp >= NB - 1) bp -= NB - 1;
    bq = t - rank;
    if (bq < 0) bq += NB - 1;
  }
}

// pair q of local round lr: all pairs of the 2B columns in block round 0
// (circle method over 2B), the B x B cross pairs (w, B + (w + lr) mod B) after
template <int B>
__device__ __forceinline__ void pair_of(int t, int lr, int q, int& i, int& j) {
  constexpr int R = 2 * B - 1;
  if (t != 0) {
    i = q;
    j = B + (q + lr) % B;
  } else if (q == 0) {
    i = R;
    j = lr;
  } else {
    i = lr + q;
    if (i >= R) i -= R;
    j = lr - q;
    if (j < 0) j += R;
  }
}

// rotation parameters of index x: x' = cs x + sp partner, new diagonal, partner
// and an active flag packed in w
__device__ __forceinline__ float4 prm(float cs, float sp, float dn, int partner, bool act) {
  return make_float4(cs, sp, dn, __int_as_float(partner | (act ? 256 : 0)));
}

}  // namespace jg

template <int EA, int EJ, int B>
__global__ void __launch_bounds__(NT32, 1) jacobi32_gram_kernel(const double* __restrict__ V, long long ldv, Dim nv_d,
                                                             Dim m_d, double* __restrict__ Jout, long long ldj,
                                                             int max_sweeps, float tol, float tol_abs, int* log) {
  constexpr int MST = 128 * EA, JST = 128 * EJ, W = 2 * B, GS = W + 1, NSL = NT32 / 32 / 2;
  // working areas.  X role: the two blocks' vectors ([MST][B] each) and their
  // B x B Gram matrices; J role: the two blocks' rotation columns ([JST][B]
  // each).  Every block is contiguous (a pull from another CTA reads whole
  // lines) and the second of a pair is offset by 16 floats (a row of 2B
  // columns then spans all 32 banks)
  constexpr int HA = MST * B + 16, HG = B * B, AREA = 2 * HA + 2 * HG;
  constexpr int HJ = JST * B + 16, JAREA = 2 * HJ;
  static_assert(B == NT32 / 32 && W == 32, "32 working columns, one per lane; one pair per warp");
  static_assert(B * MST / 4 == NT32 * EA && B * JST / 4 == NT32 * EJ, "one float4 per thread and unit");
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), CS = (int)cl.num_blocks() / 2, NB = 2 * CS;
  const bool isJ = crank >= CS;                 // the second half of the cluster keeps the rotation columns
  const int rank = isJ ? crank - CS : crank;    // the block pair this CTA follows
  extern __shared__ float4 sm4[];
  float* smf = reinterpret_cast<float*>(sm4);
  float* area = smf;                            // X role: two working areas
  float* gp = area + 2 * AREA;                  //   partial Gram matrices: NSL x W x W
  float* G = gp + NSL * W * W;                  //   W x GS
  float* Vr = G + W * GS;                       //   W x GS
  float* jarea = smf;                           // J role: two working areas
  float* vslot = jarea + 2 * JAREA;             //   the X partner's V of the last two block rounds (W x W)
  __shared__ float4 P[W];                       // rotation parameters of the current round, per index
  __shared__ int s_cnt, s_any, s_vflag[2];
  const int nv = (int)dv(nv_d), m = (int)dv(m_d);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto ja = [&](float* ar, int r, int c) -> float& { return ar[(c >> 4) * HJ + r * B + (c & 15)]; };
  // rows [0, rows) of a pair of row-major [.][B] blocks (the second hs floats
  // after the first) times the 2B x 2B rotation in vq (this lane's column)
  auto apply = [&](float* X0, int hs, int rows, const float* vq) {
    float* X1 = X0 + hs;
#pragma unroll 2
    for (int r = warp; r < rows; r += NT32 / 32) {
      const float4* x0 = reinterpret_cast<const float4*>(X0 + r * B);
      const float4* x1 = reinterpret_cast<const float4*>(X1 + r * B);
      float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
      for (int u = 0; u < W / 4; ++u) {
        const float4 v = u < B / 4 ? x0[u] : x1[u - B / 4];
        o0 = fmaf(v.x, vq[4 * u], o0);
        o1 = fmaf(v.y, vq[4 * u + 1], o1);
        o2 = fmaf(v.z, vq[4 * u + 2], o2);
        o3 = fmaf(v.w, vq[4 * u + 3], o3);
      }
      __syncwarp();
      (lane < B ? X0 : X1)[r * B + (lane & 15)] = (o0 + o1) + (o2 + o3);
    }
  };

  // block round 0 layout: vectors in X area 0, the identity in J area 0
  {
    int b0, b1;
    jg::blocks(0, rank, NB, b0, b1);
    for (int h = 0; h < 2; ++h)
      for (int k = 0; k < B; ++k) {
        const int c = (h ? b1 : b0) * B + k;
        if (!isJ)
          for (int l = tid; l < MST; l += NT32)
            area[h * HA + l * B + k] = (c < nv && l < m) ? (float)V[c * ldv + l] : 0.f;
        else
          for (int l = tid; l < JST; l += NT32) ja(jarea, l, h * B + k) = (c < nv && l == c) ? 1.f : 0.f;
      }
    if (tid == 0) s_vflag[0] = s_vflag[1] = 0;
  }
  // J role, step g: the rotation columns of block round g follow their
  // blocks (pulled from the J CTAs that held them in round g - 1) and take
  // the V that the X partner sent in round g.  Step g runs while the X CTAs
  // work on round g + 1, so it is off their critical path.
  auto jstep = [&](int g) {
    const int tg = g % (NB - 1);
    int bp, bq;
    jg::blocks(tg, rank, NB, bp, bq);
    float* cur = jarea + (g & 1) * JAREA;
    if (g > 0) {
      const int tp = tg == 0 ? NB - 2 : tg - 1;
      float4 rj[2][EJ];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int orank, oh;
        jg::owner(h ? bq : bp, tp, NB, CS, orank, oh);
        const float4* sJ =
            reinterpret_cast<const float4*>(cl.map_shared_rank(jarea + ((g - 1) & 1) * JAREA, orank + CS) + oh * HJ);
#pragma unroll
        for (int u = 0; u < EJ; ++u) rj[h][u] = sJ[tid + u * NT32];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4* dJ = reinterpret_cast<float4*>(cur + h * HJ);
#pragma unroll
        for (int u = 0; u < EJ; ++u) dJ[tid + u * NT32] = rj[h][u];
      }
      __syncthreads();
    }
    if (s_vflag[g & 1]) {
      float vq[W];
#pragma unroll
      for (int k = 0; k < W; ++k) vq[k] = vslot[(g & 1) * W * W + k * W + lane];
      apply(cur, HJ, nv < JST ? nv : JST, vq);
    }
  };

  int gr = 0, t_last = 0;  // block rounds done; block round of the last data
  int sweep = 0;
  for (sweep = 0; sweep < max_sweeps && nv >= 2; ++sweep) {
    if (tid == 0) s_cnt = 0;
    int rot = 0;  // this CTA rotated a pair in this sweep (uniform across the CTA)
    cl.sync();
    for (int t = 0; t < NB - 1; ++t, ++gr) {
      t_last = t;
      if (isJ) {
        if (gr > 0) jstep(gr - 1);
        cl.sync();
        continue;
      }
      int bp, bq;
      jg::blocks(t, rank, NB, bp, bq);
      float* cur = area + (gr & 1) * AREA;
      // 1. pull the two blocks (and after a sweep's first block round their
      //    Gram matrices) from their positions of the previous block round
      if (gr > 0) {
        const int tp = t == 0 ? NB - 2 : t - 1;
        float4 ra[2][EA];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int orank, oh;
          jg::owner(h ? bq : bp, tp, NB, CS, orank, oh);
          const float* src = cl.map_shared_rank(area + ((gr - 1) & 1) * AREA, orank);
          const float4* sA = reinterpret_cast<const float4*>(src + oh * HA);
#pragma unroll
          for (int u = 0; u < EA; ++u) ra[h][u] = sA[tid + u * NT32];
        }
        float4 rg = make_float4(0.f, 0.f, 0.f, 0.f);
        const int gh = tid / (HG / 4), gq = tid % (HG / 4);
        if (t != 0 && tid < 2 * HG / 4) {
          int orank, oh;
          jg::owner(gh ? bq : bp, tp, NB, CS, orank, oh);
          const float* src = cl.map_shared_rank(area + ((gr - 1) & 1) * AREA, orank);
          rg = reinterpret_cast<const float4*>(src + 2 * HA + oh * HG)[gq];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float4* dA = reinterpret_cast<float4*>(cur + h * HA);
#pragma unroll
          for (int u = 0; u < EA; ++u) dA[tid + u * NT32] = ra[h][u];
        }
        if (t != 0 && tid < 2 * HG / 4) reinterpret_cast<float4*>(cur + 2 * HA + gh * HG)[gq] = rg;
      }
      if (tid == 0) s_any = 0;
      __syncthreads();
      // 2. Gram matrix.  In the first block round of a sweep every entry is a
      //    fresh dot product (warp (half, slice) sums rows slice, slice + NSL,
      //    ... for G rows half*16 .. half*16+15 against column `lane`); after
      //    it only the cross block X_0^T X_1 is new, and the two diagonal
      //    blocks are the blocks' Gram matrices as the previous block round
      //    left them (rotated two-sidedly, so their errors stay relative to
      //    each entry's scale), refreshed again at the next sweep
      if (t == 0) {
        const int half = warp & 1, sl = warp >> 1;
        float acc[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) acc[p] = 0.f;
        const float* xl = cur + (lane >> 4) * HA + (lane & 15);
        const float* xh = cur + half * HA;
#pragma unroll 4
        for (int r = sl; r < m; r += NSL) {
          const float xq = xl[r * B];
          const float4* xr = reinterpret_cast<const float4*>(xh + r * B);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 v = xr[u];
            acc[4 * u + 0] = fmaf(v.x, xq, acc[4 * u + 0]);
            acc[4 * u + 1] = fmaf(v.y, xq, acc[4 * u + 1]);
            acc[4 * u + 2] = fmaf(v.z, xq, acc[4 * u + 2]);
            acc[4 * u + 3] = fmaf(v.w, xq, acc[4 * u + 3]);
          }
        }
#pragma unroll
        for (int p = 0; p < 16; ++p) gp[(sl * W + half * 16 + p) * W + lane] = acc[p];
        __syncthreads();
        for (int e = tid; e < W * W; e += NT32) {
          float g = 0.f;
#pragma unroll
          for (int sl2 = 0; sl2 < NSL; ++sl2) g += gp[sl2 * W * W + e];
          G[(e / W) * GS + e % W] = g;
        }
      } else {
        // cross block: 32 slices of rows (warp, lane half), lane & 15 the column
        // of the second block, 16 accumulators over the first block's columns
        const int sl = warp * 2 + (lane >> 4), bcol = lane & 15;
        float acc[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) acc[p] = 0.f;
#pragma unroll 2
        for (int r = sl; r < m; r += 2 * (NT32 / 32)) {
          const float xq = cur[HA + r * B + bcol];
          const float4* xr = reinterpret_cast<const float4*>(cur + r * B);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 v = xr[u];
            acc[4 * u + 0] = fmaf(v.x, xq, acc[4 * u + 0]);
            acc[4 * u + 1] = fmaf(v.y, xq, acc[4 * u + 1]);
            acc[4 * u + 2] = fmaf(v.z, xq, acc[4 * u + 2]);
            acc[4 * u + 3] = fmaf(v.w, xq, acc[4 * u + 3]);
          }
        }
#pragma unroll
        for (int p = 0; p < 16; ++p) gp[(sl * 16 + p) * 16 + bcol] = acc[p];
        __syncthreads();
        for (int e = tid; e < 3 * HG; e += NT32) {
          if (e < HG) {
            const int a = e / 16, bb = e % 16;
            float g = 0.f;
            for (int sl2 = 0; sl2 < 2 * (NT32 / 32); ++sl2) g += gp[(sl2 * 16 + a) * 16 + bb];
            G[a * GS + B + bb] = g;
            G[(B + bb) * GS + a] = g;
          } else {
            const int f = e - HG, h = f / HG, a = (f % HG) / B, bb = f % B;
            G[(h * B + a) * GS + h * B + bb] = cur[2 * HA + h * HG + a * B + bb];
          }
        }
      }
      for (int e = tid; e < W * W; e += NT32) Vr[(e / W) * GS + e % W] = (e / W == e % W) ? 1.f : 0.f;
      __syncthreads();
      // 3. the block round's rotations on G, accumulated in V.  Each round:
      //    (a) lanes 0..15 of warp 0 compute the rotations of the round's 16
      //    pairs (one lane per pair, so the transcendental unit sees each
      //    rotation once) and publish them per index; barrier; (b) warp w
      //    writes rows i, j of its pair w of R^T G R (four entries of G each,
      //    the partners' rotations from (a)) and columns i, j of V R; barrier
      const int nlr = t == 0 ? W - 1 : B;
      for (int lr = 0; lr < nlr; ++lr) {
        if (tid < B) {
          int i, j;
          jg::pair_of<B>(t, lr, tid, i, j);
          const float a = G[i * GS + i], b = G[j * GS + j], g = G[i * GS + j];
          const int gi = (i < B ? bp : bq) * B + (i % B), gj = (j < B ? bp : bq) * B + (j % B);
          const bool go = gi < nv && gj < nv && g != 0.f && fabsf(g) * rsqrtf(a) * rsqrtf(b) > tol &&
                          fabsf(g) > tol_abs * fmaxf(a, b);
          if (go) {
            const float zeta = __fdividef(b - a, 2.f * g);
            const float tt = copysignf(__fdividef(1.f, fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))), zeta);
            const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
            P[i] = jg::prm(cs, -sn, fmaxf(fmaf(-tt, g, a), 0.f), j, true);
            P[j] = jg::prm(cs, sn, fmaxf(fmaf(tt, g, b), 0.f), i, true);
            s_any = 1;
          } else {
            P[i] = jg::prm(1.f, 0.f, a, j, false);
            P[j] = jg::prm(1.f, 0.f, b, i, false);
          }
        }
        __syncthreads();
        int i, j;
        jg::pair_of<B>(t, lr, warp, i, j);
        const float4 pi = P[i];
        const bool go = (__float_as_int(pi.w) & 256) != 0;
        const float cs = pi.x, sn = -pi.y;
        {
          const float4 pl = P[lane];
          const int ql = __float_as_int(pl.w) & 255;
          const float gil = G[i * GS + lane], gjl = G[j * GS + lane];
          const float giq = G[i * GS + ql], gjq = G[j * GS + ql];
          __syncwarp();
          // rows first (this pair), then columns (the pair of `lane`)
          const float ril = fmaf(-sn, gjl, cs * gil), riq = fmaf(-sn, gjq, cs * giq);
          const float rjl = fmaf(sn, gil, cs * gjl), rjq = fmaf(sn, giq, cs * gjq);
          float ni = fmaf(pl.y, riq, pl.x * ril), nj = fmaf(pl.y, rjq, pl.x * rjl);
          if (go) {  // the pair's own 2 x 2 block in closed form
            if (lane == i) {
              ni = pi.z;
              nj = 0.f;
            } else if (lane == j) {
              ni = 0.f;
              nj = P[j].z;
            }
          }
          G[i * GS + lane] = ni;
          G[j * GS + lane] = nj;
          if (go) {
            const float vi = Vr[lane * GS + i], vj = Vr[lane * GS + j];
            Vr[lane * GS + i] = fmaf(-sn, vj, cs * vi);
            Vr[lane * GS + j] = fmaf(sn, vi, cs * vj);
          }
        }
        __syncthreads();
      }
      // the blocks' rotated Gram matrices travel with them to the next block round
      for (int e = tid; e < 2 * HG; e += NT32) {
        const int h = e / HG, a = (e % HG) / B, bb = e % B;
        cur[2 * HA + h * HG + a * B + bb] = G[(h * B + a) * GS + h * B + bb];
      }
      // 4. X <- X V when something rotated, and V to the J partner
      if (s_any) {
        rot = 1;
        float vq[W];
#pragma unroll
        for (int k = 0; k < W; ++k) vq[k] = Vr[k * GS + lane];
        apply(cur, HA, m, vq);
        float* vs = cl.map_shared_rank(vslot + (gr & 1) * W * W, crank + CS);
        for (int e = tid; e < W * W; e += NT32) vs[e] = Vr[(e / W) * GS + e % W];
      }
      if (tid == 0) *cl.map_shared_rank(&s_vflag[gr & 1], crank + CS) = s_any;
      if (t == NB - 2 && rot && tid == 0) s_cnt = 1;  // a flag, not a count: only zero matters
      cl.sync();
    }
    int total = 0;
    for (int r = 0; r < CS; ++r) total += *cl.map_shared_rank(&s_cnt, r);
    cl.sync();  // every CTA has read the flags before the next sweep resets them
    if (total == 0) break;
  }
  // the rotation columns of the last block round, then no CTA leaves while
  // another may still read its shared memory
  if (isJ && gr > 0) jstep(gr - 1);
  cl.sync();
  if (log && crank == 0 && tid == 0) {
    log[0] = nv;
    log[1] = m;
    log[2] = sweep + 1;
  }
  if (isJ) {
    int b0, b1;
    jg::blocks(t_last, rank, NB, b0, b1);
    float* fin = jarea + (gr > 0 ? (gr - 1) & 1 : 0) * JAREA;
    for (int h = 0; h < 2; ++h)
      for (int k = 0; k < B; ++k) {
        const int c = (h ? b1 : b0) * B + k;
        if (c >= nv) continue;
        for (int l = tid; l < nv; l += NT32) Jout[(long long)c * ldj + l] = (double)ja(fin, l, h * B + k);
      }
  }
}

// H = 1.5 I - 0.5 G  (the Newton-Schulz factor)
__global__ void ns_factor_kernel(const double* G, double* H, long long ld, Dim n_d) {
  const long long n = dv(n_d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    H[i * ld + j] = -0.5 * G[i * ld + j] + (i == j ? 1.5 : 0.0);
  }
}

// Omega_ji = G_ij / (G_ii - G_jj): the first-order angle of the pair (i, j)
// that zeroes G_ij (Omega is antisymmetric).  Pairs whose angle is not small
// (nearly equal values) are left alone.
__device__ __forceinline__ double omega_angle(const double* G, long long ld, long long i, long long j) {
  const double gij = G[i * ld + j], den = G[i * ld + i] - G[j * ld + j];
  if (den == 0.0) return 0.0;
  const double th = gij / den;
  return fabs(th) <= 0.1 ? th : 0.0;
}

// Angles above kSmallAngle only occur between nearly equal values (in
// practice inside the noise floor of the spectrum); they are the ones damped.
constexpr double kSmallAngle = 1e-3;

// rs[i] = sum over j of |Omega_ji| (= |Omega_ij|) with |Omega_ji| > kSmallAngle, one block per row
__global__ void omega_rowsum_kernel(const double* G, long long ld, Dim n_d, double* rs) {
  const long long n = dv(n_d);
  __shared__ double red[32];
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    double a = 0.0;
    for (long long j = threadIdx.x; j < n; j += blockDim.x)
      if (j != i) {
        const double th = fabs(omega_angle(G, ld, i, j));
        if (th > kSmallAngle) a += th;
      }
    a = block_sum(a, red);
    if (threadIdx.x == 0) rs[i] = a;
  }
}

// M = I + Omega'^T.  Angles up to kSmallAngle are kept as they are (with at
// most 512 vectors their row sums stay below 0.52); larger ones are scaled by
// min(1, 1/(4 max(rs_i, rs_j))), so their row sums stay below 1/4.  Omega' is
// antisymmetric, so ||Omega'||_2 <= 0.77 and ||I + Omega'||_2 <= 1.26 <
// sqrt(3): the Newton-Schulz iteration that follows always converges.  Without
// the damping, clusters of near-equal tiny values can give ||I + Omega|| > 2
// and the iteration diverges.
__global__ void omega_kernel(const double* G, const double* rs, double* M, long long ld, Dim n_d) {
  const long long n = dv(n_d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    double v = 1.0;
    if (i != j) {
      // M[i][j] = Omega'_ji
      v = omega_angle(G, ld, i, j);
      const double r = fmax(rs[i], rs[j]);
      if (fabs(v) > kSmallAngle && r > 0.25) v *= 0.25 / r;
    }
    M[i * ld + j] = v;
  }
}

// norms[c] = |W[c]| over m entries (rows of W, ld ldw)
__global__ void row_norms_kernel(const double* W, long long ldw, Dim n_d, Dim m_d, double* norms) {
  const long long n = dv(n_d), m = dv(m_d);
  __shared__ double red[32];
  for (long long c = blockIdx.x; c < n; c += gridDim.x) {
    double s = 0.0;
    for (long long l = threadIdx.x; l < m; l += blockDim.x) {
      const double x = W[c * ldw + l];
      s = fma(x, x, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) norms[c] = sqrt(s);
  }
}

// Householder QR with column pivoting (Businger & Golub 1965) of a small
// matrix A (nr x nc, nr <= MR) in one thread-block cluster, FP32, for the
// preconditioned Jacobi of the mixed SVD (Drmac & Veselic 2008): the rows of
// R1 in A P = Q1 R1 are graded, and one-sided Jacobi on them needs far fewer
// sweeps than on the columns of an unpivoted R.  A[a][i] = Ain[a * lda + i]
// (A is the transpose of a column-major R0).  Column i lives in the shared
// memory of CTA i % CS; a step is one cluster barrier to publish every CTA's
// best remaining norm, one to publish the reflector, and a warp per column
// applying it and recomputing that column's remaining norm.  Outputs: R1
// (k1 x nc, pivoted column order) row-major at R1 (row stride ldr1), the thin
// Q1 (nr x k1) row-major at Q1 (row stride ldq), k1 = min(nr, nc) at *k1_out.
// Vg: global scratch of k1 * MR floats for the reflectors.
template <int MR>
__global__ void __launch_bounds__(NT32) qrcp_cluster_kernel(const double* __restrict__ Ain, long long lda,
                                                            Dim nr_d, Dim nc_d, int cpc, double* R1, long long ldr1,
                                                            double* Q1, long long ldq, float* Vg, int* k1_out) {
  constexpr int PER = MR / 32;  // rows per lane
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CS = (int)cl.num_blocks();
  extern __shared__ float smf[];
  float* col = smf;                              // cpc columns of MR floats
  float* nrm = col + (long long)cpc * MR;        // remaining squared norms (-1: chosen)
  float* s_v = nrm + cpc;                        // reflector of the current step
  float* s_v2 = s_v + MR;                        // second reflector buffer (forming Q1)
  float* s_tau = s_v2 + MR;                      // tau of every step
  int* s_piv = reinterpret_cast<int*>(s_tau + MR);  // logical -> physical column (<= NT32 columns)
  int* s_pos = s_piv + NT32;                     // physical -> logical
  __shared__ float s_cval, s_btau;
  __shared__ int s_cidx, s_p;
  const int nr = (int)dv(nr_d), nc = (int)dv(nc_d), k1 = nr < nc ? nr : nc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT32 / 32;

  for (int sl = warp; sl < cpc; sl += nw) {
    const int c = rank + sl * CS;
    float s2 = 0.f;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int a = lane + 32 * t;
      const float x = (c < nc && a < nr) ? (float)Ain[(long long)a * lda + c] : 0.f;
      col[sl * MR + a] = x;
      s2 = fmaf(x, x, s2);
    }
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) nrm[sl] = c < nc ? s2 : -1.f;
  }
  __syncthreads();

  for (int j = 0; j < k1; ++j) {
    // this CTA's best remaining column (ties: smaller index)
    if (warp == 0) {
      float bv = -1.f;
      int bi = -1;
      for (int sl = lane; sl < cpc; sl += 32)
        if (nrm[sl] > bv) {
          bv = nrm[sl];
          bi = rank + sl * CS;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_cval = bv;
        s_cidx = bi;
      }
    }
    cl.sync();
    if (warp == 0) {  // the same pivot in every CTA
      float bv = -1.f;
      int bi = -1;
      if (lane < CS) {
        bv = *cl.map_shared_rank(&s_cval, lane);
        bi = *cl.map_shared_rank(&s_cidx, lane);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_p = bi;
        s_piv[j] = bi;
      }
    }
    __syncthreads();
    const int p = s_p;
    const int owner = p < 0 ? -1 : p % CS;
    if (owner == rank && warp == 0) {  // form reflector j from column p
      float* x = col + (p / CS) * MR;
      float s2 = 0.f;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        if (a > j && a < nr) s2 = fmaf(x[a], x[a], s2);
      }
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      const float alpha = x[j];
      float tj = 0.f, beta = alpha, sc = 0.f;
      if (s2 != 0.f) {
        const float nr2 = sqrtf(alpha * alpha + s2);
        beta = alpha >= 0.f ? -nr2 : nr2;
        tj = (beta - alpha) / beta;
        sc = 1.f / (alpha - beta);
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        float v = 0.f;
        if (a == j) v = 1.f;
        else if (a > j && a < nr) {
          v = x[a] * sc;
          x[a] = v;
        }
        s_v[a] = v;
        Vg[(long long)j * MR + a] = v;
      }
      if (lane == 0) {
        x[j] = beta;
        s_btau = tj;
        nrm[p / CS] = -1.f;
      }
    }
    cl.sync();
    if (owner >= 0 && owner != rank) {
      const float* rv = cl.map_shared_rank(s_v, owner);
      for (int a = tid; a < MR; a += NT32) s_v[a] = rv[a];
      if (tid == 0) s_tau[j] = *cl.map_shared_rank(&s_btau, owner);
    } else if (tid == 0) {
      s_tau[j] = s_btau;
    }
    __syncthreads();
    const float tj = s_tau[j];
    for (int sl = warp; sl < cpc; sl += nw) {
      if (nrm[sl] < 0.f) continue;
      float* y = col + sl * MR;
      float d = 0.f;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        if (a >= j) d = fmaf(s_v[a], y[a], d);
      }
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      const float w = tj * d;
      float s2 = 0.f;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        if (a >= j) {
          const float yn = fmaf(-w, s_v[a], y[a]);
          y[a] = yn;
          if (a > j && a < nr) s2 = fmaf(yn, yn, s2);
        }
      }
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm[sl] = s2;
    }
    __syncthreads();
  }
  // columns never chosen (nc > nr) follow in ascending order; inverse order
  if (tid == 0) {  // a permutation whatever the norms were (non-finite input included)
    for (int c = 0; c < nc; ++c) s_pos[c] = -1;
    for (int q = 0; q < k1; ++q) {
      const int c = s_piv[q];
      if (c >= 0 && c < nc && s_pos[c] < 0) s_pos[c] = q;
      else s_piv[q] = -1;
    }
    int nxt = 0;
    for (int q = 0; q < nc; ++q)
      if (q >= k1 || s_piv[q] < 0) {
        while (nxt < nc && s_pos[nxt] >= 0) ++nxt;
        if (nxt >= nc) break;
        s_piv[q] = nxt;
        s_pos[nxt] = q;
      }
    if (rank == 0 && k1_out) *k1_out = k1;
  }
  __syncthreads();
  for (int sl = warp; sl < cpc; sl += nw) {
    const int c = rank + sl * CS;
    if (c >= nc) continue;
    const int pos = s_pos[c];
    if (pos < 0 || pos >= nc) continue;
    for (int r = lane; r < k1; r += 32) R1[(long long)r * ldr1 + pos] = r <= pos ? (double)col[sl * MR + r] : 0.0;
  }
  __threadfence();
  cl.sync();  // every reflector is in Vg and every CTA is done with its columns
  // thin Q1: column q = H_0 ... H_{k1-1} e_q, for q = rank, rank + CS, ...
  for (int sl = warp; sl < cpc; sl += nw) {
    const int q = rank + sl * CS;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int a = lane + 32 * t;
      col[sl * MR + a] = (a == q) ? 1.f : 0.f;
    }
  }
  // reflectors come from L2 one step ahead (a register per thread) into two
  // alternating shared buffers: one CTA barrier per reflector
  static_assert(MR <= NT32, "one reflector element per thread");
  float nxt = (tid < MR && k1 > 0) ? __ldcg(Vg + (long long)(k1 - 1) * MR + tid) : 0.f;
  for (int j = k1 - 1; j >= 0; --j) {
    float* vb = (j & 1) ? s_v2 : s_v;
    if (tid < MR) vb[tid] = nxt;
    __syncthreads();
    if (j > 0 && tid < MR) nxt = __ldcg(Vg + (long long)(j - 1) * MR + tid);
    const float tj = s_tau[j];
    for (int sl = warp; sl < cpc; sl += nw) {
      const int q = rank + sl * CS;
      if (q >= k1 || q < j) continue;  // H_j leaves e_q alone for q < j
      float* y = col + sl * MR;
      float d = 0.f;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        if (a >= j) d = fmaf(vb[a], y[a], d);
      }
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      const float w = tj * d;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int a = lane + 32 * t;
        if (a >= j) y[a] = fmaf(-w, vb[a], y[a]);
      }
    }
  }
  __syncthreads();
  for (int sl = warp; sl < cpc; sl += nw) {
    const int q = rank + sl * CS;
    if (q >= k1) continue;
    for (int a = lane; a < nr; a += 32) Q1[(long long)a * ldq + q] = (double)col[sl * MR + a];
  }
}

// Order key of a pivot candidate, in integer arithmetic (the FP64 pipe of
// this part is narrow, comparisons and divisions included): monotone in the
// value, a NaN above everything, 0 for no candidate.
__device__ __forceinline__ unsigned long long piv_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b & 0x7fffffffffffffffULL) > 0x7ff0000000000000ULL) return ~0ULL;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

// (ak, ai) ranks above (bk, bi): the larger key, then the smaller index
__device__ __forceinline__ bool piv_better(unsigned long long ak, int ai, unsigned long long bk, int bi) {
  return ak > bk || (ak == bk && ai >= 0 && (bi < 0 || ai < bi));
}

// Cholesky factorisation with diagonal pivoting (Higham, Accuracy and
// Stability of Numerical Algorithms, 2nd ed., Sec. 10.3) of a symmetric
// positive semidefinite G (n x n, n <= MN, FP64) in one thread-block cluster.
// Step k picks the largest remaining diagonal entry d = S_pp of the Schur
// complement S, emits row k of R, u = S[:, p] / sqrt(d) (zero at the indices
// already chosen, u_p = sqrt(d)), and subtracts u u^T from S.  The result
// satisfies R^T R = G up to the dropped remainder: R is the triangular factor
// of a QR with column pivoting of any M with M^T M = G, with its columns
// left in their original order (R P is upper trapezoidal).  It stops after
// kcap rows, or once d <= n 2^-52 d_0 (d_0: the first pivot), the level at
// which S holds only the rounding of G; k >= 1 rows are always written.
// Column c of S lives in the shared memory of CTA c % CS; lane s of warp 0
// keeps the diagonal entry of the CTA's s-th column in a register.  A step:
// every warp picks the pivot from the candidates (key, index, sqrt(d),
// 1/sqrt(d)) that all CTAs pushed into this CTA's slots (one per CTA, two
// alternating slot sets), each thread reads its entry of the pivot column
// from the owner's shared memory (chosen columns are never written again),
// warp 0 updates the diagonal and pushes this CTA's next candidate to every
// CTA while the others update the owned columns, one thread per row; one
// cluster barrier.  Outputs: R (k x n) row-major with row stride ldr, k at
// *k_out.
template <int MN>
__global__ void __launch_bounds__(MN) pchol_cluster_kernel(const double* __restrict__ G, long long ldg, Dim n_d,
                                                           Dim kcap_d, int cpc, double* R, long long ldr,
                                                           int* k_out) {
  static_assert(MN % 32 == 0 && MN >= 32, "whole warps");
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CS = (int)cl.num_blocks();
  extern __shared__ double smd[];
  double* col = smd;                     // cpc columns of MN doubles
  double* u = col + (long long)cpc * MN;  // the current row of R
  // candidates pushed by the CTAs of the cluster: key, index, sqrt(d), 1/sqrt(d)
  __shared__ unsigned long long s_ck[2][16];
  __shared__ int s_ci[2][16];
  __shared__ double s_cr[2][16], s_cq[2][16];
  __shared__ int s_done[MN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long nl = dv(n_d), kc = dv(kcap_d);
  const int n = (int)(nl < MN ? nl : MN);
  const int kmax = (int)(kc < n ? kc : n);
  s_done[tid] = tid >= n;
  for (int sl = 0; sl < cpc; ++sl) {
    const int c = rank + sl * CS;
    col[sl * MN + tid] = (c < n && tid < n) ? G[(long long)c * ldg + tid] : 0.0;
  }
  // warp 0, lane s < cpc: the diagonal entry of owned column s
  const int myc = rank + lane * CS;
  const bool mine = warp == 0 && lane < cpc && myc < n;
  double dg = mine ? G[(long long)myc * ldg + myc] : 0.0;
  // best remaining owned diagonal entry, pushed into slot set b of every CTA
  auto push = [&](int b) {
    unsigned long long bk = 0;
    int bi = -1;
    double bv = 0.0;
    if (mine && !s_done[myc]) {
      bk = piv_key(dg);
      bi = myc;
      bv = dg;
    }
    for (int o = 16; o > 0; o >>= 1) {  // every lane ends with the best
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (piv_better(ok, oi, bk, bi)) {
        bk = ok;
        bi = oi;
        bv = ov;
      }
    }
    double r = 0.0, q = 0.0;
    if (lane == 0 && bi >= 0) {  // NaN stays NaN; d <= 0 (rounding) gives a zero row
      r = bv > 0.0 ? sqrt(bv) : (bv == bv ? 0.0 : bv);
      q = r != 0.0 ? 1.0 / r : 0.0;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (lane < CS) {
      *cl.map_shared_rank(&s_ck[b][rank], lane) = bk;
      *cl.map_shared_rank(&s_ci[b][rank], lane) = bi;
      *cl.map_shared_rank(&s_cr[b][rank], lane) = r;
      *cl.map_shared_rank(&s_cq[b][rank], lane) = q;
    }
  };
  cl.sync();  // every CTA of the cluster runs before any distributed access
  if (warp == 0) push(0);
  cl.sync();
  unsigned long long thr = 0;  // stop key: n 2^-52 d_0 (none when d_0 is NaN)
  int k = 0;
  for (; k < kmax; ++k) {
    const int b = k & 1;
    unsigned long long key = 0;  // the same pivot in every warp of every CTA
    int p = -1, from = lane;
    if (lane < CS) {
      key = s_ck[b][lane];
      p = s_ci[b][lane];
    }
    for (int o = 16; o > 0; o >>= 1) {  // every lane: the loop exit is uniform
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int oi = __shfl_xor_sync(0xffffffffu, p, o);
      const int of = __shfl_xor_sync(0xffffffffu, from, o);
      if (piv_better(ok, oi, key, p)) {
        key = ok;
        p = oi;
        from = of;
      }
    }
    if (p < 0) break;
    if (k == 0) {
      if (key != ~0ULL) {
        const double r0 = s_cr[b][from];
        thr = piv_key((double)n * 0x1p-52 * (r0 * r0));
      }
    } else if (key <= thr) {
      break;
    }
    const double r = s_cr[b][from], q = s_cq[b][from];
    const double* pc = cl.map_shared_rank(col, p % CS) + (long long)(p / CS) * MN;
    double ui = 0.0;
    if (tid == p) ui = r;
    else if (tid < n && !s_done[tid]) ui = pc[tid] * q;
    u[tid] = ui;
    if (tid < n && rank == k % CS) R[(long long)k * ldr + tid] = ui;
    if (tid == p) s_done[p] = 1;
    __syncthreads();
    if (warp == 0) {
      if (mine && !s_done[myc]) dg = fma(-u[myc], u[myc], dg);
      push(b ^ 1);
    }
#pragma unroll
    for (int sl = 0; sl < 16; ++sl) {
      const int c = rank + sl * CS;
      if (sl >= cpc || c >= n || s_done[c]) continue;
      col[sl * MN + tid] = fma(-ui, u[c], col[sl * MN + tid]);
    }
    cl.sync();
  }
  if (k == 0 && kmax > 0) {  // no pivot at all (n = 0 cannot reach here): a zero row
    if (rank == 0 && tid < n) R[tid] = 0.0;
    k = 1;
  }
  if (rank == 0 && tid == 0 && k_out) *k_out = k;
  cl.sync();  // no CTA leaves while another may still read its columns
}

// J[c][a] = W[c][a] / norms[c] (0 where the norm is 0): unit rows
__global__ void scale_rows_kernel(const double* W, long long ldw, const double* norms, Dim rows_d, Dim cols_d,
                                  double* J, long long ldj) {
  const long long rows = dv(rows_d), cols = dv(cols_d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * cols;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / cols, a = e % cols;
    const double nc = norms[c];
    J[c * ldj + a] = nc != 0.0 ? W[c * ldw + a] / nc : 0.0;
  }
}

inline int eg(long long total) {
  long long g = (total + 255) / 256;
  return (int)std::max(1LL, std::min(g, device_sms() * 8LL));
}

}  // namespace

// FP32 cluster Jacobi: J (nv x nv, vector-major, ld ldj) from nv FP64 vectors
// V (length m, ld ldv).  Sizes nvmax, mmax pick the cluster and smem layout.
template <int EA, int EJ>
static cudaError_t launch_j32(cudaLaunchConfig_t* cfg, const double* V, long long ldv, Dim nv, Dim m, double* J,
                              long long ldj, int cpc, int* log) {
  // FP32 stops an order of magnitude above its rounding floor; the FP64
  // refinement squares the remaining non-orthogonality twice
  const int max_sweeps = 20;
  const float tol = 1e-4f, tol_abs = 1e-6f;
  return cudaLaunchKernelEx(cfg, jacobi32_cluster_kernel<EA, EJ>, V, ldv, nv, m, J, ldj, cpc, max_sweeps, tol, tol_abs,
                            log);
}

// dynamic shared memory of jacobi32_gram_kernel: the larger of the X role
// (two working areas with the blocks' Gram matrices, partial Gram matrices,
// G and V) and the J role (two working areas, two V slots)
static size_t jg_smem(int EA, int EJ) {
  constexpr int B = NT32 / 32, W = 2 * B, NSL = NT32 / 32 / 2;
  const size_t xr = (size_t)2 * (2 * (128 * EA * B + 16) + 2 * B * B) + (size_t)NSL * W * W + 2 * (size_t)W * (W + 1);
  const size_t jr = (size_t)2 * (2 * (128 * EJ * B + 16)) + 2 * (size_t)W * W;
  return std::max(xr, jr) * sizeof(float);
}

template <int EA, int EJ>
static size_t j32_smem(int cpc, int CS) {
  return (size_t)cpc * 128 * (EA + EJ) * sizeof(float) + 2 * (size_t)cpc * CS * sizeof(void*);
}

// FP32 cluster Jacobi: J (nv x nv, vector-major, ld ldj) from nv FP64 vectors
// V (length m, ld ldv).  Sizes nvmax, mmax pick the cluster and smem layout:
// about one pair per warp per round (16 warps per CTA), at most 16 CTAs.
cudaError_t jacobi32_cluster(qtt_ctx* ctx, const double* V, long long ldv, Dim nv, Dim m, long long nvmax,
                             long long mmax, double* J, long long ldj) {
  const int EA = (int)((mmax + 127) / 128), EJ = (int)((nvmax + 127) / 128);
  if (EA > 4 || EJ > 4) return cudaErrorInvalidValue;
  int CS = 1;
  while (CS < 16 && (nvmax + 1) / 2 > (long long)CS * (NT32 / 32)) CS *= 2;
  const long long budget = 200 * 1024;
  while (CS < 16 && (long long)((nvmax + CS - 1) / CS) * 128 * (EA + EJ) * 4 > budget) CS *= 2;
  const int cpc = (int)((nvmax + CS - 1) / CS);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(NT32);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int* log = jacobi_log_slot(ctx);
  const int key = EA * 10 + EJ;
  // block kernel: 2*CS blocks of 16 columns, 4 blocks of shared memory per CTA
  {
    constexpr int Bk = NT32 / 32;
    int CSb = 1;
    while (CSb < 16 && 2LL * CSb * Bk < nvmax) CSb *= 2;
    const size_t sm_b = jg_smem(EA, EJ);
    if (2LL * CSb * Bk >= nvmax && CSb <= 8 && sm_b <= (size_t)budget && (EA == EJ) && EA <= 2) {
      // CSb CTAs rotate the vectors, CSb more keep the rotation columns
      cfg.gridDim = dim3(2 * CSb);
      at[0].val.clusterDim.x = 2 * CSb;
      cfg.dynamicSmemBytes = sm_b;
      const int max_sweeps = 20;
      const float tol = 1e-4f, tol_abs = 1e-6f;
      if (EA == 1)
        return cudaLaunchKernelEx(&cfg, jacobi32_gram_kernel<1, 1, Bk>, V, ldv, nv, m, J, ldj, max_sweeps, tol,
                                  tol_abs, log);
      return cudaLaunchKernelEx(&cfg, jacobi32_gram_kernel<2, 2, Bk>, V, ldv, nv, m, J, ldj, max_sweeps, tol, tol_abs,
                                log);
    }
  }
#define J32_CASE(a, b)                                          \
  case a * 10 + b:                                              \
    cfg.dynamicSmemBytes = j32_smem<a, b>(cpc, CS);              \
    if (cfg.dynamicSmemBytes > (size_t)budget) return cudaErrorInvalidValue; \
    return launch_j32<a, b>(&cfg, V, ldv, nv, m, J, ldj, cpc, log);
  switch (key) {
    J32_CASE(1, 1) J32_CASE(2, 2) J32_CASE(3, 3) J32_CASE(4, 4)
    J32_CASE(1, 2) J32_CASE(2, 1) J32_CASE(2, 3) J32_CASE(3, 2) J32_CASE(3, 4) J32_CASE(4, 3)
    J32_CASE(1, 3) J32_CASE(1, 4) J32_CASE(2, 4) J32_CASE(3, 1) J32_CASE(4, 1) J32_CASE(4, 2)
    default:
      return cudaErrorInvalidValue;
  }
#undef J32_CASE
}

cudaError_t ns_factor(const double* G, double* H, long long ld, Dim n, long long nmax, cudaStream_t st) {
  ns_factor_kernel<<<eg(nmax * nmax), 256, 0, st>>>(G, H, ld, n);
  return cudaGetLastError();
}

cudaError_t omega_factor(const double* G, double* rs, double* M, long long ld, Dim n, long long nmax,
                         cudaStream_t st) {
  omega_rowsum_kernel<<<(int)std::max(1LL, std::min(nmax, device_sms() * 4LL)), 256, 0, st>>>(G, ld, n, rs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  omega_kernel<<<eg(nmax * nmax), 256, 0, st>>>(G, rs, M, ld, n);
  return cudaGetLastError();
}

static size_t qrcp_smem(int cpc) {
  return ((size_t)cpc * 256 + cpc + 3 * 256) * sizeof(float) + 2 * (size_t)NT32 * sizeof(int);
}

cudaError_t qrcp_cluster(qtt_ctx* ctx, const double* Ain, long long lda, Dim nr, Dim nc, long long nmax, double* R1,
                         long long ldr1, double* Q1, long long ldq, float* Vg, int* k1_out) {
  if (nmax > 256) return cudaErrorInvalidValue;
  // at most 16 columns per CTA (one per warp), at most 16 CTAs
  const int CS = (int)std::min<long long>(16, std::max<long long>(1, (nmax + 15) / 16));
  const int cpc = (int)((nmax + CS - 1) / CS);
  if (cpc > 16) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(NT32);
  cfg.stream = ctx->stream;
  cfg.dynamicSmemBytes = qrcp_smem(cpc);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel<256>, Ain, lda, nr, nc, cpc, R1, ldr1, Q1, ldq, Vg, k1_out);
}

static size_t pchol_smem(int cpc) { return ((size_t)cpc * 256 + 256) * sizeof(double); }

cudaError_t pchol_cluster(qtt_ctx* ctx, const double* G, long long ldg, Dim n, Dim kcap, long long nmax, double* R,
                          long long ldr, int* k_out) {
  if (nmax > 256 || nmax < 1) return cudaErrorInvalidValue;
  // at most 16 columns per CTA, at most 16 CTAs (8 CTAs of 32 columns
  // measured slower: the step is bound by latency, not by the FP64 pipe)
  const int CS = (int)std::min<long long>(16, std::max<long long>(1, (nmax + 15) / 16));
  const int cpc = (int)((nmax + CS - 1) / CS);
  if (cpc > 16) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(256);
  cfg.stream = ctx->stream;
  cfg.dynamicSmemBytes = pchol_smem(cpc);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pchol_cluster_kernel<256>, G, ldg, n, kcap, cpc, R, ldr, k_out);
}

cudaError_t scale_rows(const double* W, long long ldw, const double* norms, Dim rows, Dim cols, long long rmax,
                       long long cmax, double* J, long long ldj, cudaStream_t st) {
  scale_rows_kernel<<<eg(rmax * cmax), 256, 0, st>>>(W, ldw, norms, rows, cols, J, ldj);
  return cudaGetLastError();
}

cudaError_t row_norms(const double* W, long long ldw, Dim n, Dim m, long long nmax, double* norms, cudaStream_t st) {
  row_norms_kernel<<<(int)std::max(1LL, std::min(nmax, device_sms() * 4LL)), 256, 0, st>>>(W, ldw, n, m, norms);
  return cudaGetLastError();
}

template <int EA, int EJ>
static cudaError_t init_j32() {
  const void* k = (const void*)jacobi32_cluster_kernel<EA, EJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <int EA, int EJ>
static cudaError_t init_jb() {
  const void* k = (const void*)jacobi32_gram_kernel<EA, EJ, NT32 / 32>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

static cudaError_t init_qrcp() {
  const void* k = (const void*)qrcp_cluster_kernel<256>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qrcp_smem(16));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

static cudaError_t init_pchol() {
  const void* k = (const void*)pchol_cluster_kernel<256>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pchol_smem(16));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t mixed_init() {
  cudaError_t (*fs[])() = {init_qrcp, init_pchol, init_jb<1, 1>, init_jb<2, 2>,init_j32<1, 1>, init_j32<2, 2>, init_j32<3, 3>, init_j32<4, 4>, init_j32<1, 2>,
                           init_j32<2, 1>, init_j32<2, 3>, init_j32<3, 2>, init_j32<3, 4>, init_j32<4, 3>,
                           init_j32<1, 3>, init_j32<1, 4>, init_j32<2, 4>, init_j32<3, 1>, init_j32<4, 1>,
                           init_j32<4, 2>};
  for (auto f : fs) {
    cudaError_t e = f();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qtt
