// Partial contraction of TTs of different orders over mode pairs (n_t, m_t)
// (Eq. 8 applied to each pair; Example 1's x_3^2 when the modes sit at the
// ends of the trains), chain layout.  The paired modes of X form a block at
// one end of X, those of Y a block at one end of Y, met in the same order
// walking both trains from their ends.  An operand whose block is the
// trailing one is read backwards with its rank legs swapped (a "view"), so
// both blocks lead; the sweep then runs with a separate orientation per
// operand (SweepParams::transposed / transposed_y) and the chain is emitted
// as for a leading block: X's free cores walked back (legs swapped), the
// boundary core C = X'_s joined with K, Y's free cores.  When X has no free
// mode the operands exchange roles: the environment is then K^T, the chain
// is Y's free cores walked back with C = Y'_s joined with K^T last (its right
// rank is X's end rank, 1).
#include <string.h>

#include <algorithm>

#include "host_plan.h"

namespace ttc {

// One operand as a view: core j of the view is core `orig` of the operand,
// read forwards or with its legs swapped.
struct View {
  const tt_desc* d;
  int rev;
  int n;
  int orig(int j) const { return rev ? n - 1 - j : j; }
  int rl(int j) const { return rev ? d->ranks[n - j] : d->ranks[j]; }
  int rr(int j) const { return rev ? d->ranks[n - 1 - j] : d->ranks[j + 1]; }
  int mode(int j) const { return d->modes[orig(j)]; }
};

struct PairsPlan {
  View a, b;        // a plays X's part in the chain (its free cores walked back), b Y's
  int swapped;      // a is Y (X has no free mode)
  int s;            // pairs
  int order;        // output cores
  int modes[2 * kMaxOrder];
  int ranks[2 * kMaxOrder + 1];
  int perm[2 * kMaxOrder];
};

static int pairs_plan(const tt_desc* x, const tt_desc* y, int n_pairs, const int32_t* xm, const int32_t* ym,
                      PairsPlan* pp) {
  int rc = check_desc(x);
  if (rc != TT_OK) return rc;
  rc = check_desc(y);
  if (rc != TT_OK) return rc;
  if (x->dtype != y->dtype) return TT_ERR_DTYPE;
  if (xm == nullptr || ym == nullptr || n_pairs < 1) return TT_ERR_ARG;
  const int nx = x->order, ny = y->order, s = n_pairs;
  if (s > nx || s > ny) return TT_ERR_ARG;
  if (s == nx && s == ny) return TT_ERR_ARG;  // every mode contracted: tt_contract_full
  int y_of[kMaxOrder];
  bool usedx[kMaxOrder] = {false}, usedy[kMaxOrder] = {false};
  for (int k = 0; k < nx; ++k) y_of[k] = -1;
  for (int t = 0; t < s; ++t) {
    if (xm[t] < 0 || xm[t] >= nx || ym[t] < 0 || ym[t] >= ny || usedx[xm[t]] || usedy[ym[t]]) return TT_ERR_ARG;
    usedx[xm[t]] = usedy[ym[t]] = true;
    y_of[xm[t]] = ym[t];
    if (x->modes[xm[t]] != y->modes[ym[t]]) return TT_ERR_SHAPE;
  }
  // the blocks: leading (walked 0, 1, ...) or trailing (walked N-1, N-2, ...)
  auto block = [](const bool* used, int n, int s, bool* lead, bool* trail) {
    *lead = *trail = true;
    for (int k = 0; k < n; ++k) {
      if (used[k] != (k < s)) *lead = false;
      if (used[k] != (k >= n - s)) *trail = false;
    }
  };
  bool xl, xt, yl, yt;
  block(usedx, nx, s, &xl, &xt);
  block(usedy, ny, s, &yl, &yt);
  int found = 0, rev_x = 0, rev_y = 0;
  for (int rx = 0; rx < 2 && !found; ++rx) {
    if ((rx == 0 && !xl) || (rx == 1 && !xt)) continue;
    for (int ry = 0; ry < 2 && !found; ++ry) {
      if ((ry == 0 && !yl) || (ry == 1 && !yt)) continue;
      bool ok = true;
      for (int t = 0; t < s && ok; ++t) {
        const int xk = rx ? nx - 1 - t : t, yk = ry ? ny - 1 - t : t;
        ok = y_of[xk] == yk;
      }
      if (ok) {
        found = 1;
        rev_x = rx;
        rev_y = ry;
      }
    }
  }
  if (!found) return TT_ERR_LAYOUT;
  View vx{x, rev_x, nx}, vy{y, rev_y, ny};
  pp->s = s;
  pp->swapped = nx == s ? 1 : 0;
  pp->a = pp->swapped ? vy : vx;
  pp->b = pp->swapped ? vx : vy;
  const View& A = pp->a;
  const View& B = pp->b;
  const int fa = A.n - s, fb = B.n - s;  // free modes (fa >= 1)
  pp->order = fa + fb;
  int q = 0;
  // A's free cores walked back (legs swapped), the last of them C
  for (int j = A.n - 1; j >= s; --j, ++q) {
    pp->modes[q] = A.mode(j);
    pp->ranks[q] = A.rr(j);
  }
  for (int j = s; j < B.n; ++j, ++q) {
    pp->modes[q] = B.mode(j);
    pp->ranks[q] = B.rl(j);
  }
  pp->ranks[pp->order] = 1;
  // perm: axis p of the chain is axis perm[p] of Eq. 8's Z (X's free modes
  // ascending, then Y's)
  auto x_rank = [&](int orig) {  // position of X's free mode `orig` among X's free modes
    int r = 0;
    for (int k = 0; k < orig; ++k) r += usedx[k] ? 0 : 1;
    return r;
  };
  auto y_rank = [&](int orig) {
    int r = 0;
    for (int k = 0; k < orig; ++k) r += usedy[k] ? 0 : 1;
    return r;
  };
  const int fx = nx - s;
  q = 0;
  for (int j = A.n - 1; j >= s; --j, ++q) {
    const int o = A.orig(j);
    pp->perm[q] = pp->swapped ? fx + y_rank(o) : x_rank(o);
  }
  for (int j = s; j < B.n; ++j, ++q) {
    const int o = B.orig(j);
    pp->perm[q] = pp->swapped ? x_rank(o) : fx + y_rank(o);
  }
  return TT_OK;
}

// Sweep parameters: the s paired modes of both views, then the emission of C
// and the free-core copies.
static int build_pairs(const PairsPlan& pp, const tt_desc* z, int64_t* z_log2_dev, int32_t* status_dev,
                       SweepParams* out) {
  SweepParams& p = *out;
  memset(&p, 0, sizeof(p));
  const View& A = pp.a;
  const View& B = pp.b;
  const int s = pp.s;
  p.n_steps = s;
  p.transposed = A.rev;
  p.transposed_y = B.rev;
  for (int j = 0; j < s; ++j) {
    SweepStep& st = p.step[j];
    st.gx = A.d->cores[A.orig(j)];
    st.gy = B.d->cores[B.orig(j)];
    st.I = A.mode(j);
    st.rin_x = A.rl(j);
    st.rout_x = A.rr(j);
    st.rin_y = B.rl(j);
    st.rout_y = B.rr(j);
  }
  p.rx0 = 1;
  p.ry0 = 1;
  p.final_scalar = 0;
  p.renorm_bits = A.d->dtype == TT_F64 ? kRenormBitsF64 : kRenormBitsF32;
  p.status = status_dev;
  EmitParams& ep = p.emit;
  ep.enabled = 1;
  const int ob = A.orig(s);
  ep.gx = A.d->cores[ob];
  ep.ra = A.d->ranks[ob];
  ep.I = A.d->modes[ob];
  ep.rb = A.d->ranks[ob + 1];
  ep.lead = A.rev ? 0 : 1;
  ep.ry = B.rl(s);
  const int fa = A.n - s;
  ep.c_out = z->cores[fa - 1];
  ep.z_log2_out = z_log2_dev;
  auto add = [&](const void* src, void* dst, int r0, int I, int r1, int swap) -> int {
    if (!swap && src == dst) return TT_OK;  // output aliases its input: nothing to copy
    if (swap && src == dst) return TT_ERR_ARG;
    if (ep.n_copies >= kMaxCopies) return TT_ERR_TOO_LARGE;
    if (static_cast<int64_t>(r0) * I * r1 >= (int64_t(1) << 31)) return TT_ERR_TOO_LARGE;
    CopyTask& t = ep.copy[ep.n_copies++];
    t.src = src;
    t.dst = dst;
    t.r0 = r0;
    t.I = I;
    t.r1 = r1;
    t.swap = swap;
    return TT_OK;
  };
  int rc = TT_OK;
  int q = 0;
  // A'_j^T for j = A.n-1 .. s+1: a swapped copy of a forward view's core, a
  // plain copy of a reversed one's
  for (int j = A.n - 1; j > s && rc == TT_OK; --j, ++q) {
    const int o = A.orig(j);
    rc = add(A.d->cores[o], z->cores[q], A.d->ranks[o], A.d->modes[o], A.d->ranks[o + 1], A.rev ? 0 : 1);
  }
  ++q;  // C
  for (int j = s; j < B.n && rc == TT_OK; ++j, ++q) {
    const int o = B.orig(j);
    rc = add(B.d->cores[o], z->cores[q], B.d->ranks[o], B.d->modes[o], B.d->ranks[o + 1], B.rev ? 1 : 0);
  }
  return rc;
}

}  // namespace ttc

using namespace ttc;

extern "C" int tt_pairs_shape(const tt_desc* x, const tt_desc* y, int n_pairs, const int32_t* xmodes,
                              const int32_t* ymodes, int32_t* z_order, int32_t* z_modes, int32_t* z_ranks,
                              int32_t* z_perm) {
  if (z_order == nullptr || z_modes == nullptr || z_ranks == nullptr || z_perm == nullptr) return TT_ERR_ARG;
  PairsPlan pp;
  const int rc = pairs_plan(x, y, n_pairs, xmodes, ymodes, &pp);
  if (rc != TT_OK) return rc;
  *z_order = pp.order;
  for (int q = 0; q < pp.order; ++q) {
    z_modes[q] = pp.modes[q];
    z_ranks[q] = pp.ranks[q];
    z_perm[q] = pp.perm[q];
  }
  z_ranks[pp.order] = 1;
  return TT_OK;
}

extern "C" int tt_contract_pairs(const tt_desc* x, const tt_desc* y, int n_pairs, const int32_t* xmodes,
                                 const int32_t* ymodes, int prec, const tt_desc* z, int64_t* z_log2_dev,
                                 int32_t* status_dev, tt_stream stream) {
  PairsPlan pp;
  int rc = pairs_plan(x, y, n_pairs, xmodes, ymodes, &pp);
  if (rc != TT_OK) return rc;
  const bool tf32 = prec == TT_P_TF32X3 || prec == TT_P_TF32;
  if (prec != TT_P_NATIVE && !tf32) return TT_ERR_UNSUPPORTED;
  if (x->dtype == TT_BF16) return TT_ERR_UNSUPPORTED;
  if (tf32 && x->dtype != TT_F32) return TT_ERR_DTYPE;
  rc = check_desc(z);
  if (rc != TT_OK) return rc;
  if (z->order != pp.order || z->dtype != x->dtype) return TT_ERR_SHAPE;
  for (int q = 0; q < pp.order; ++q)
    if (z->modes[q] != pp.modes[q] || z->ranks[q] != pp.ranks[q] || z->ranks[q + 1] != pp.ranks[q + 1])
      return TT_ERR_SHAPE;
  SweepParams p;
  rc = build_pairs(pp, z, z_log2_dev, status_dev, &p);
  if (rc != TT_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (tf32) {
    if (sweep_max_rank(p) > kTf32MaxRank) return TT_ERR_UNSUPPORTED;
    const int C = tf32_cluster_size(pow2_floor(std::min(16, sweep_max_mode(p))));
    if (C < 1) return TT_ERR_CUDA;
    return launch_tf32_sweep(p, prec == TT_P_TF32X3, C, s) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  return launch_sweep(p, x->dtype, s);
}
