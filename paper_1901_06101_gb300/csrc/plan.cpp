// Host planning of an H-BACA call over one or many blocks (trees, leaves,
// merge stages, workspace layout).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "types.h"

namespace hbaca {

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t cur = 0;
  Region take(size_t bytes) {
    Region r;
    r.off = cur;
    r.bytes = bytes;
    cur = align_up(cur + std::max<size_t>(bytes, 1));
    return r;
  }
};

// BACA shared-memory footprint (mirrors baca_smem_bytes in baca.cuh).
size_t baca_smem(size_t esz, int mr, int nc, int d) {
  size_t w = std::max((size_t)mr * d, (size_t)d * nc);
  size_t b = w * esz;
  b += (size_t)(2 * d + d + 2 * d * d + d) * esz;
  b += (size_t)d * 8;
  b += 2 * 16 + 32 * 8 + 32 * 4 + 96 * 8;
  b += (size_t)(4 * d + 16) * 4;
  b += (size_t)mr + nc + std::max(mr, nc) + 64;
  return b;
}

bool check_gen(const hbaca_gen& g, std::string& err) {
  if (g.m < 1 || g.n < 1 || g.m >= (1ll << 31) || g.n >= (1ll << 31)) { err = "m and n must be in [1, 2^31)"; return false; }
  if (g.dtype != HBACA_F64 && g.dtype != HBACA_C128) { err = "unknown dtype"; return false; }
  switch (g.kind) {
    case HBACA_GEN_DENSE:
      if (!g.a || g.lda < g.m) { err = "DENSE needs a and lda >= m"; return false; }
      break;
    case HBACA_GEN_GAUSSIAN:
      if (g.dtype != HBACA_F64) { err = "GAUSSIAN is float64"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 64 || !(g.h > 0.0 && std::isfinite(g.h))) {
        err = "GAUSSIAN needs x, y, 1 <= dim <= 64 and a finite h > 0";
        return false;
      }
      break;
    case HBACA_GEN_HELMHOLTZ:
      if (g.dtype != HBACA_C128) { err = "HELMHOLTZ is complex128"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 64 || !std::isfinite(g.k)) {
        err = "HELMHOLTZ needs x, y, 1 <= dim <= 64 and a finite k";
        return false;
      }
      break;
    case HBACA_GEN_SPARSE_PRODUCT:
      if (g.dtype != HBACA_F64) { err = "SPARSE_PRODUCT is float64"; return false; }
      if (!g.p_rowptr || !g.p_colidx || !g.p_val || !g.q_colptr || !g.q_rowidx || !g.q_val || g.K < 0 ||
          g.r2 < 0 || g.r2 > 16 || (g.r2 > 0 && (!g.p2 || !g.q2))) {
        err = "SPARSE_PRODUCT needs CSR P, CSC Q and 0 <= r2 <= 16 (with p2, q2)";
        return false;
      }
      break;
    case HBACA_GEN_LOWRANK:
      if (!g.lu || !g.lv || g.lr < 0) { err = "LOWRANK needs lu, lv, lr >= 0"; return false; }
      break;
    case HBACA_GEN_POLYNOMIAL:
      if (g.dtype != HBACA_F64) { err = "POLYNOMIAL is float64"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 1024 || !std::isfinite(g.h)) {
        err = "POLYNOMIAL needs x, y, 1 <= dim <= 1024 and a finite h";
        return false;
      }
      break;
    case HBACA_GEN_HANKEL2D:
      if (g.dtype != HBACA_C128) { err = "HANKEL2D is complex128"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 64 || !(g.k > 0.0 && std::isfinite(g.k))) {
        err = "HANKEL2D needs x, y, 1 <= dim <= 64 and a finite k > 0";
        return false;
      }
      break;
    default:
      err = "unknown generator kind";
      return false;
  }
  return true;
}

}  // namespace

std::vector<std::vector<Span>> tree_levels(int64_t n, int L) {
  std::vector<std::vector<Span>> lv(L + 1);
  lv[L] = {Span(0, n)};
  for (int l = L; l > 0; --l) {
    for (const Span& s : lv[l]) {
      int64_t a = (s.second + 1) / 2;
      lv[l - 1].push_back(Span(s.first, a));
      lv[l - 1].push_back(Span(s.first + a, s.second - a));
    }
  }
  return lv;
}

int block_levels(int64_t m, int64_t n, int levels) {
  int L = levels;
  if (levels < 0) {
    const int64_t target = -(int64_t)levels;
    L = 0;
    while ((std::max(m, n) + (1ll << L) - 1) / (1ll << L) > target) ++L;
    while (L > 0 && (1ll << L) > std::min(m, n)) --L;
    return L;
  }
  if ((1ll << L) > std::min(m, n)) return -1;
  return L;
}

bool make_plan(const hbaca_gen* gens, int nblocks, const hbaca_opts& o, int sms, Plan& p, std::string& err) {
  if (!gens || nblocks < 1) { err = "need at least one block"; return false; }
  for (int b = 0; b < nblocks; ++b) {
    if (!check_gen(gens[b], err)) { err = "block " + std::to_string(b) + ": " + err; return false; }
    if (gens[b].kind != gens[0].kind || gens[b].dtype != gens[0].dtype) {
      err = "all blocks must share the generator kind and dtype";
      return false;
    }
  }
  if (nblocks > 1 && gens[0].kind != HBACA_GEN_GAUSSIAN) {
    err = "batched compression is available for the GAUSSIAN generator";
    return false;
  }
  if (!(o.eps > 0.0 && o.eps < 1.0)) { err = "eps must be in (0, 1)"; return false; }
  if (o.d < 1 || o.d > 32) { err = "d must be in [1, 32]"; return false; }
  if (o.flags & ~(HBACA_FLAG_ASYNC | HBACA_FLAG_PROFILE | HBACA_FLAG_TAPE | HBACA_FLAG_GRAPH | HBACA_FLAG_SINGLE_CLUSTER |
                  HBACA_FLAG_FROB)) {
    err = "unknown option flags";
    return false;
  }
  if (!(o.srrqr_f == 0.0 || (o.srrqr_f > 1.0 && o.srrqr_f < 1e150))) {
    err = "srrqr_f must be 0 or a finite value > 1"; return false;
  }
  if (o.levels > 12 || o.levels < -(1 << 30)) { err = "levels out of range"; return false; }
  if (o.cluster != 0 && (o.cluster < 1 || o.cluster > 16 || (o.cluster & (o.cluster - 1)))) {
    err = "cluster must be 0 or a power of two <= 16";
    return false;
  }
  if (o.rank_cap < 0 || o.leaf_rank_cap < 0) { err = "rank caps must be >= 0"; return false; }
  if (o.rank_cap > 1024 || o.leaf_rank_cap > 1024) { err = "rank caps must be <= 1024"; return false; }
  if (sms <= 0) sms = 152;
  p.gens.assign(gens, gens + nblocks);
  p.opts = o;
  p.cplx = gens[0].dtype == HBACA_C128;
  p.esz = p.cplx ? 16 : 8;
  p.d = o.d;
  p.nblocks = nblocks;
  p.Lb.resize(nblocks);
  p.cap_b.resize(nblocks);
  p.Lmax = 0;
  for (int b = 0; b < nblocks; ++b) {
    const int L = block_levels(gens[b].m, gens[b].n, o.levels);
    if (L < 0) {
      err = "block " + std::to_string(b) + ": levels L needs 2^L <= min(m, n)";
      return false;
    }
    p.Lb[b] = L;
    p.Lmax = std::max(p.Lmax, L);
    const int64_t mn = std::min(gens[b].m, gens[b].n);
    p.cap_b[b] = o.rank_cap ? std::min<int64_t>(o.rank_cap, mn) : std::min<int64_t>(mn, 1024);
    p.rank_cap_max = std::max(p.rank_cap_max, p.cap_b[b]);
  }

  // ---- leaves (block by block, row-major over the leaf grid)
  std::vector<LeafDesc> leaves;
  std::vector<std::vector<std::vector<Span>>> rows(nblocks), cols(nblocks);
  p.leaf_first.assign(nblocks, 0);
  int64_t uo = 0, vo = 0, to = 0, tdo = 0;
  const int rec = 4 + 3 * p.d;
  for (int b = 0; b < nblocks; ++b) {
    rows[b] = tree_levels(gens[b].m, p.Lb[b]);
    cols[b] = tree_levels(gens[b].n, p.Lb[b]);
    p.leaf_first[b] = (int)leaves.size();
    const int nb = 1 << p.Lb[b];
    for (int a = 0; a < nb; ++a)
      for (int c = 0; c < nb; ++c) {
        LeafDesc L;
        std::memset(&L, 0, sizeof(L));
        L.row0 = rows[b][0][a].first;
        L.col0 = cols[b][0][c].first;
        L.m = (int32_t)rows[b][0][a].second;
        L.n = (int32_t)cols[b][0][c].second;
        int64_t lc = o.leaf_rank_cap ? o.leaf_rank_cap : 1024;
        L.rcap = (int32_t)std::min<int64_t>(std::min<int64_t>(L.m, L.n), lc);
        L.tape_iters = std::min(L.m, L.n);
        L.stream_id = ((int64_t)b << 24) | ((int64_t)a << 12) | c;
        L.u_off = uo;
        L.v_off = vo;
        L.tape_off = to;
        L.taped_off = tdo;
        L.block = b;
        uo += (int64_t)L.m * L.rcap;
        vo += (int64_t)L.rcap * L.n;
        to += (int64_t)L.tape_iters * rec;
        tdo += (int64_t)L.tape_iters * 2;
        p.mmax = std::max(p.mmax, L.m);
        p.nmax = std::max(p.nmax, L.n);
        p.rcap_max = std::max(p.rcap_max, L.rcap);
        leaves.push_back(L);
      }
  }
  p.nleaves = (int)leaves.size();
  // processing order: largest leaves first, so the persistent clusters finish together
  std::vector<int32_t> order(p.nleaves);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return (int64_t)leaves[x].m * leaves[x].n > (int64_t)leaves[y].m * leaves[y].n;
  });

  // ---- BACA cluster size.  The persistent clusters (about sms / c of them)
  // take the leaves in ceil(leaves / clusters) rounds of a leaf time that
  // falls as 1 / c (the leaf work is FP64-bound and split over the cluster's
  // SMs): pick the c in 1, 2, 4, 8 with the fewest rounds / c, ties to the
  // smaller, at least 16 rows per CTA; shared memory within budget.
  int c = o.cluster;
  if (c == 0) {
    c = 1;
    const int64_t s_eff = std::max(sms, 1);
    double best = 1e300;
    for (int cc = 1; cc <= 8; cc *= 2) {
      if (cc > 1 && (p.mmax + cc - 1) / cc < 16) break;
      const int64_t clusters = std::max<int64_t>(1, s_eff / cc);
      const double cost = (double)((p.nleaves + clusters - 1) / clusters) / cc;
      if (cost < best * (1.0 - 1e-9)) {
        best = cost;
        c = cc;
      }
    }
  }
  while (baca_smem(p.esz, (p.mmax + c - 1) / c, (p.nmax + c - 1) / c, p.d) > 200 * 1024 && c < 16) c *= 2;
  p.baca_cluster = c;
  p.mr_max = (p.mmax + c - 1) / c;
  p.nc_max = (p.nmax + c - 1) / c;
  p.baca_smem = baca_smem(p.esz, p.mr_max, p.nc_max, p.d);
  if (p.baca_smem > 227 * 1024) { err = "leaf too large for shared memory even with 16-CTA clusters"; return false; }
  {
    size_t per_sm = std::min<size_t>(8, std::max<size_t>(1, (228 * 1024) / (p.baca_smem + 1024)));
    p.max_clusters_scratch = (int)std::max<int64_t>(1, std::min<int64_t>(p.nleaves, (int64_t)sms * per_sm / c));
  }
  p.cscr_stride = (int64_t)p.mmax * p.d;
  p.rscr_stride = (int64_t)p.d * p.nmax;
  p.gscr_stride = (int64_t)2 * c * p.rcap_max * p.d;

  // ---- block references: full store (after the vertical merge of level l),
  // half store (after the horizontal merge of level l), one result per block;
  // every reference's rank lives at its own index of one rank array
  // (with HBACA_FLAG_TAPE no store is reused across levels, and every node
  // keeps all singular triplets of its core: storage capacity = the producing
  // task's k capacity, the number stored goes to a second rank-array slot)
  p.tape = (o.flags & HBACA_FLAG_TAPE) != 0;
  p.frob = (o.flags & HBACA_FLAG_FROB) != 0;
  std::vector<int64_t> kc_b(nblocks);
  for (int b = 0; b < nblocks; ++b) kc_b[b] = std::min<int64_t>(2 * p.cap_b[b], 2 * std::min(gens[b].m, gens[b].n));
  std::vector<BlockRef> refs;
  int ntaped = 0;
  p.full_idx.assign(nblocks, std::vector<std::vector<int>>(p.Lmax + 1));
  p.half_idx.assign(nblocks, std::vector<std::vector<int>>(p.Lmax + 1));
  size_t full_u = 0, full_s = 0, full_v = 0, half_u = 0, half_s = 0, half_v = 0;
  auto add_ref = [&](int64_t m, int64_t n, int64_t cap, int64_t store_cap, int64_t& u, int64_t& s, int64_t& v) {
    BlockRef r;
    std::memset(&r, 0, sizeof(r));
    r.m = (int32_t)m;
    r.n = (int32_t)n;
    r.u_off = u; r.s_off = s; r.v_off = v;
    r.ldu = m; r.ldv = n;
    r.rank_slot = (int32_t)refs.size();
    r.cap = (int32_t)cap;
    r.store_cap = (int32_t)(p.tape ? std::max(store_cap, cap) : cap);
    r.full_slot = p.tape ? -2 - ntaped++ : -1;  // resolved once the number of refs is known
    u += m * r.store_cap; s += r.store_cap; v += r.store_cap * n;
    refs.push_back(r);
    return (int)refs.size() - 1;
  };
  int64_t fu = 0, fs = 0, fv = 0, hu = 0, hs = 0, hv = 0;  // running offsets (tape)
  for (int l = 0; l < p.Lmax; ++l) {  // full store level l: blocks with L_b > l
    int64_t u = p.tape ? fu : 0, s = p.tape ? fs : 0, v = p.tape ? fv : 0;
    for (int b = 0; b < nblocks; ++b) {
      if (p.Lb[b] <= l) continue;
      const int nr = (int)rows[b][l].size(), ncn = (int)cols[b][l].size();
      p.full_idx[b][l].assign(nr * ncn, -1);
      for (int a = 0; a < nr; ++a)
        for (int cc = 0; cc < ncn; ++cc) {
          const int64_t sc = l == 0 ? leaves[p.leaf_first[b] + a * ncn + cc].rcap : kc_b[b];
          p.full_idx[b][l][a * ncn + cc] =
              add_ref(rows[b][l][a].second, cols[b][l][cc].second, p.cap_b[b], sc, u, s, v);
        }
    }
    fu = u; fs = s; fv = v;
    full_u = std::max<size_t>(full_u, u); full_s = std::max<size_t>(full_s, s); full_v = std::max<size_t>(full_v, v);
  }
  for (int l = 1; l <= p.Lmax; ++l) {  // half store level l: blocks with L_b >= l
    int64_t u = p.tape ? hu : 0, s = p.tape ? hs : 0, v = p.tape ? hv : 0;
    for (int b = 0; b < nblocks; ++b) {
      if (p.Lb[b] < l) continue;
      const int nr = (int)rows[b][l - 1].size(), ncn = (int)cols[b][l].size();
      p.half_idx[b][l].assign(nr * ncn, -1);
      for (int a = 0; a < nr; ++a)
        for (int cc = 0; cc < ncn; ++cc)
          p.half_idx[b][l][a * ncn + cc] =
              add_ref(rows[b][l - 1][a].second, cols[b][l][cc].second, p.cap_b[b], kc_b[b], u, s, v);
    }
    hu = u; hs = s; hv = v;
    half_u = std::max<size_t>(half_u, u); half_s = std::max<size_t>(half_s, s); half_v = std::max<size_t>(half_v, v);
  }
  p.user_ref_first = (int)refs.size();
  for (int b = 0; b < nblocks; ++b) {
    int64_t z = 0, z2 = 0, z3 = 0;
    const int keep = ntaped;
    add_ref(gens[b].m, gens[b].n, p.cap_b[b], p.cap_b[b], z, z2, z3);
    refs.back().store_cap = (int32_t)p.cap_b[b];
    refs.back().full_slot = -1;  // the caller's buffers hold the kept triplets only
    ntaped = keep;
  }
  if (p.tape) {  // root node of every block, in the full store after all levels
    p.root_tape_first = (int)refs.size();
    int64_t u = fu, s = fs, v = fv;
    for (int b = 0; b < nblocks; ++b) {
      const int64_t sc = p.Lb[b] == 0 ? leaves[p.leaf_first[b]].rcap : kc_b[b];
      add_ref(gens[b].m, gens[b].n, p.cap_b[b], sc, u, s, v);
    }
    full_u = std::max<size_t>(full_u, u); full_s = std::max<size_t>(full_s, s); full_v = std::max<size_t>(full_v, v);
  }
  p.nrefs = (int)refs.size();
  for (BlockRef& r : refs)
    if (r.full_slot <= -2) r.full_slot = p.nrefs + (-r.full_slot - 2);
  p.nslots = p.nrefs + ntaped;

  // ---- tasks, grouped into chunks whose scratch (QR operands, cores) fits the
  // budget; scratch offsets are local to a chunk, chunks run one after another
  p.task_storage.clear();
  p.stages.clear();
  size_t qr_elems = 0, tau_elems = 0, core_elems = 0, ord_elems = 0;
  const size_t budget = (size_t)8 << 30;  // bytes of chunk scratch
  auto add_stage = [&](std::vector<SvdTask>& all, int kind, int in_store, int out_store) {
    size_t i = 0;
    while (i < all.size()) {
      std::vector<SvdTask> ch;
      int64_t ao = 0, tauo = 0, co = 0, oo = 0;
      int rmax = 0, kmx = 0;
      while (i < all.size()) {
        SvdTask t = all[i];
        const int64_t kc = t.kcap;
        const int64_t need_qr = (int64_t)t.rows_a * kc * (t.a_in_baca ? 0 : 1) + (int64_t)t.rows_b * kc;
        const size_t bytes = (size_t)(ao + need_qr + co + 5 * kc * kc + tauo + 3 * kc) * p.esz + (size_t)(oo + 2 * kc) * 4;
        if (!ch.empty() && bytes > budget) break;
        if (!t.a_in_baca) { t.a_off = ao; ao += (int64_t)t.rows_a * kc; }
        if (t.kind == TASK_LEAF) { t.b_off = ao; ao += (int64_t)t.rows_b * kc; }
        t.tau_off = tauo; tauo += 3 * kc;
        t.m_off = co; co += kc * kc;
        t.y_off = co; co += kc * kc;
        t.x_off = co; co += kc * kc;
        t.xs_off = co; co += kc * kc;
        t.ys_off = co; co += kc * kc;
        t.ord_off = oo; oo += 2 * kc;
        rmax = std::max(rmax, std::max(t.rows_a, t.rows_b));
        kmx = std::max<int>(kmx, (int)kc);
        ch.push_back(t);
        ++i;
      }
      qr_elems = std::max<size_t>(qr_elems, (size_t)ao);
      tau_elems = std::max<size_t>(tau_elems, (size_t)tauo);
      core_elems = std::max<size_t>(core_elems, (size_t)co);
      ord_elems = std::max<size_t>(ord_elems, (size_t)oo);
      Stage st;
      st.kind = kind;
      st.ntasks = (int)ch.size();
      st.kcap = kmx;
      st.rows_max = rmax;
      st.in_store = in_store;
      st.out_store = out_store;
      p.task_storage.push_back(ch);
      p.stages.push_back(st);
    }
  };
  {
    std::vector<SvdTask> ts(p.nleaves);
    for (int i = 0; i < p.nleaves; ++i) {
      const LeafDesc& L = leaves[i];
      const int b = L.block;
      const int nb = 1 << p.Lb[b];
      const int a = (i - p.leaf_first[b]) / nb, cc = (i - p.leaf_first[b]) % nb;
      SvdTask& t = ts[i];
      std::memset(&t, 0, sizeof(t));
      t.kind = TASK_LEAF;
      t.kcap = L.rcap;
      t.in1 = i;
      t.a_off = L.u_off;
      t.src_u_off = L.u_off;
      t.a_in_baca = p.tape ? 0 : 1;  // a tape keeps the BACA factors for the reverse pass
      t.rows_a = L.m;
      t.lda = L.m;
      t.rows_b = L.n;
      t.src_v_off = L.v_off;
      t.out = p.Lb[b] == 0 ? (p.tape ? p.root_tape_first + b : p.user_ref_first + b) : p.full_idx[b][0][a * nb + cc];
      t.trunc = p.frob ? 2 * p.Lb[b] + 1 : 0;
    }
    add_stage(ts, TASK_LEAF, -1, 0);
  }
  for (int l = 1; l <= p.Lmax; ++l) {
    std::vector<SvdTask> th, tv;
    for (int b = 0; b < nblocks; ++b) {
      if (p.Lb[b] < l) continue;
      const int64_t kc = std::min<int64_t>(2 * p.cap_b[b], 2 * std::min(gens[b].m, gens[b].n));
      {  // horizontal: row nodes at level l-1, column nodes at level l
        const int nr = (int)rows[b][l - 1].size(), ncn = (int)cols[b][l].size(), ncp = (int)cols[b][l - 1].size();
        for (int a = 0; a < nr; ++a)
          for (int cc = 0; cc < ncn; ++cc) {
            SvdTask t;
            std::memset(&t, 0, sizeof(t));
            t.kind = TASK_HORIZ;
            t.kcap = (int32_t)kc;
            t.in1 = p.full_idx[b][l - 1][a * ncp + 2 * cc];
            t.in2 = p.full_idx[b][l - 1][a * ncp + 2 * cc + 1];
            t.rows_a = (int32_t)rows[b][l - 1][a].second;
            t.lda = t.rows_a;
            t.out = p.half_idx[b][l][a * ncn + cc];
            t.m1 = (int32_t)cols[b][l - 1][2 * cc].second;
            t.trunc = p.frob ? 2 * p.Lb[b] + 1 : 0;
            th.push_back(t);
          }
      }
      {  // vertical: row and column nodes at level l; children in the half store
        const int nr = (int)rows[b][l].size(), ncn = (int)cols[b][l].size();
        for (int a = 0; a < nr; ++a)
          for (int cc = 0; cc < ncn; ++cc) {
            SvdTask t;
            std::memset(&t, 0, sizeof(t));
            t.kind = TASK_VERT;
            t.kcap = (int32_t)kc;
            t.in1 = p.half_idx[b][l][(2 * a) * ncn + cc];
            t.in2 = p.half_idx[b][l][(2 * a + 1) * ncn + cc];
            t.rows_a = (int32_t)cols[b][l][cc].second;
            t.lda = t.rows_a;
            t.out = p.Lb[b] == l ? (p.tape ? p.root_tape_first + b : p.user_ref_first + b)
                                 : p.full_idx[b][l][a * ncn + cc];
            t.m1 = (int32_t)rows[b][l - 1][2 * a].second;
            t.trunc = p.frob ? 2 * p.Lb[b] + 1 : 0;
            tv.push_back(t);
          }
      }
    }
    add_stage(th, TASK_HORIZ, 0, 1);
    add_stage(tv, TASK_VERT, 1, 0);
  }
  for (size_t i = 0; i < p.stages.size(); ++i) p.stages[i].tasks_h = &p.task_storage[i];

  // ---- descriptor staging (host-written)
  std::vector<char>& D = p.desc;
  D.clear();
  auto put = [&](const void* src, size_t bytes) {
    size_t off = D.size();
    D.resize(align_up(off + bytes));
    if (bytes) std::memcpy(D.data() + off, src, bytes);
    return off;
  };
  p.leafdesc_off = put(leaves.data(), leaves.size() * sizeof(LeafDesc));
  p.order_off = put(order.data(), order.size() * sizeof(int32_t));
  {
    std::vector<GaussBlockParams> gp(nblocks);
    for (int b = 0; b < nblocks; ++b) {
      gp[b].x = gens[b].x;
      gp[b].y = gens[b].y;
      gp[b].dim = gens[b].dim;
      gp[b].pad = 0;
      gp[b].c = gens[b].h > 0.0 ? -1.0 / (2.0 * gens[b].h * gens[b].h) : 0.0;
    }
    p.gparams_off = put(gp.data(), gp.size() * sizeof(GaussBlockParams));
  }
  p.refs_off = put(refs.data(), refs.size() * sizeof(BlockRef));
  for (size_t si = 0; si < p.stages.size(); ++si) {
    Stage& st = p.stages[si];
    const std::vector<SvdTask>& ts = *st.tasks_h;
    st.tasks_off = put(ts.data(), ts.size() * sizeof(SvdTask));
    std::vector<QrJob> qj;
    std::vector<QJob> aj;
    for (int i = 0; i < st.ntasks; ++i) {
      qj.push_back(QrJob{i, 0});
      if (st.kind == TASK_LEAF) qj.push_back(QrJob{i, 1});
      QJob a{};
      a.task = i;
      a.which = 0;
      a.to_v = st.kind == TASK_VERT ? 1 : 0;
      aj.push_back(a);
      if (st.kind == TASK_LEAF) {
        QJob bq{};
        bq.task = i;
        bq.which = 1;
        bq.to_v = 1;
        aj.push_back(bq);
      }
    }
    st.nqr = (int)qj.size();
    st.nq = (int)aj.size();
    st.qrjobs_off = put(qj.data(), qj.size() * sizeof(QrJob));
    st.qjobs_off = put(aj.data(), aj.size() * sizeof(QJob));
  }

  // ---- workspace layout
  Layout Lo;
  p.status = Lo.take(64);
  p.queue = Lo.take(64);
  p.desc_region = Lo.take(D.size());
  p.leafout_off = Lo.take((size_t)p.nleaves * sizeof(LeafOut)).off;
  p.ranks_off = Lo.take((size_t)p.nslots * 4).off;
  for (Stage& st : p.stages) st.dims_off = Lo.take((size_t)st.ntasks * sizeof(TaskDims)).off;
  p.uar = Lo.take((size_t)uo * p.esz);
  p.var = Lo.take((size_t)vo * p.esz);
  p.cscr = Lo.take((size_t)p.max_clusters_scratch * p.cscr_stride * p.esz);
  p.rscr = Lo.take((size_t)p.max_clusters_scratch * p.rscr_stride * p.esz);
  p.gscr = Lo.take((size_t)p.max_clusters_scratch * p.gscr_stride * p.esz);
  p.tape_int = Lo.take((size_t)to * 4);
  p.tape_dbl = Lo.take((size_t)tdo * 8);
  p.full_u = Lo.take(full_u * p.esz);
  p.full_s = Lo.take(full_s * 8);
  p.full_v = Lo.take(full_v * p.esz);
  p.half_u = Lo.take(half_u * p.esz);
  p.half_s = Lo.take(half_s * 8);
  p.half_v = Lo.take(half_v * p.esz);
  p.qr = Lo.take(qr_elems * p.esz);
  p.tau = Lo.take(tau_elems * p.esz);
  p.core = Lo.take(core_elems * p.esz);
  p.ord = Lo.take(ord_elems * 4);
  {
    size_t tot = 1;
    for (Stage& st : p.stages) {
      st.jlist_off = tot - 1;
      tot += (size_t)st.ntasks;
    }
    p.jlist = Lo.take(tot * 4);
  }
  {
    int kx = (int)p.rank_cap_max;
    for (const Stage& st : p.stages) kx = std::max(kx, st.kcap);
    p.xplen = 2 + 2 * kx;
    p.xpart = Lo.take((size_t)kXSlots * 2 * (size_t)p.xplen * p.esz);
    p.xcnt = Lo.take((size_t)kXSlots * 4);
  }
  p.total = Lo.cur;
  return true;
}

void bind_user_result(Plan& p, int b, const hbaca_result& r) {
  BlockRef u;
  const size_t off = p.refs_off + (size_t)(p.user_ref_first + b) * sizeof(BlockRef);
  std::memcpy(&u, p.desc.data() + off, sizeof(u));
  u.ldu = r.ldu;
  u.ldv = r.ldv;
  u.U = r.U;
  u.S = r.S;
  u.V = r.V;
  std::memcpy(p.desc.data() + off, &u, sizeof(u));
}

}  // namespace hbaca
