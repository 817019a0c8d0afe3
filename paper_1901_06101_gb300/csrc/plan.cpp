// Host planning of an H-BACA call (trees, leaves, merge stages, workspace).
#include "plan.h"

#include <algorithm>
#include <cstring>

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
  b += 2 * 16 + 32 * 8 + 32 * 4 + 64 * 8;
  b += (size_t)(4 * d + 16) * 4;
  b += (size_t)mr + nc + std::max(mr, nc) + 64;
  return b;
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

static bool check_gen(const hbaca_gen& g, std::string& err) {
  if (g.m < 1 || g.n < 1 || g.m >= (1ll << 31) || g.n >= (1ll << 31)) { err = "m and n must be in [1, 2^31)"; return false; }
  if (g.dtype != HBACA_F64 && g.dtype != HBACA_C128) { err = "unknown dtype"; return false; }
  switch (g.kind) {
    case HBACA_GEN_DENSE:
      if (!g.a || g.lda < g.m) { err = "DENSE needs a and lda >= m"; return false; }
      break;
    case HBACA_GEN_GAUSSIAN:
      if (g.dtype != HBACA_F64) { err = "GAUSSIAN is float64"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 64 || !(g.h > 0.0)) { err = "GAUSSIAN needs x, y, 1 <= dim <= 64, h > 0"; return false; }
      break;
    case HBACA_GEN_HELMHOLTZ:
      if (g.dtype != HBACA_C128) { err = "HELMHOLTZ is complex128"; return false; }
      if (!g.x || !g.y || g.dim < 1 || g.dim > 64) { err = "HELMHOLTZ needs x, y, 1 <= dim <= 64"; return false; }
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
    default:
      err = "unknown generator kind";
      return false;
  }
  return true;
}

bool make_plan(const hbaca_gen& g, const hbaca_opts& o, int sms, Plan& p, std::string& err) {
  if (!check_gen(g, err)) return false;
  if (!(o.eps > 0.0 && o.eps < 1.0)) { err = "eps must be in (0, 1)"; return false; }
  if (o.d < 1 || o.d > 32) { err = "d must be in [1, 32]"; return false; }
  if (o.levels < 0 || o.levels > 12 || (1ll << o.levels) > std::min(g.m, g.n)) {
    err = "levels L needs 0 <= L <= 12 and 2^L <= min(m, n)";
    return false;
  }
  if (o.cluster != 0 && (o.cluster < 1 || o.cluster > 16 || (o.cluster & (o.cluster - 1)))) {
    err = "cluster must be 0 or a power of two <= 16";
    return false;
  }
  if (o.rank_cap < 0 || o.leaf_rank_cap < 0) { err = "rank caps must be >= 0"; return false; }
  if (sms <= 0) sms = 152;
  p.gen = g;
  p.opts = o;
  p.cplx = g.dtype == HBACA_C128;
  p.esz = p.cplx ? 16 : 8;
  p.L = o.levels;
  p.d = o.d;
  p.m = g.m;
  p.n = g.n;
  const int64_t mn = std::min(g.m, g.n);
  p.rank_cap = o.rank_cap ? std::min<int64_t>(o.rank_cap, mn) : std::min<int64_t>(mn, 1024);
  p.rows = tree_levels(g.m, p.L);
  p.cols = tree_levels(g.n, p.L);
  const int nb = 1 << p.L;
  p.nleaves = nb * nb;

  // ---- leaves
  std::vector<LeafDesc> leaves(p.nleaves);
  int64_t uo = 0, vo = 0, to = 0, tdo = 0;
  const int rec = 4 + 3 * p.d;
  for (int a = 0; a < nb; ++a)
    for (int b = 0; b < nb; ++b) {
      LeafDesc& L = leaves[a * nb + b];
      L.row0 = p.rows[0][a].first;
      L.col0 = p.cols[0][b].first;
      L.m = (int32_t)p.rows[0][a].second;
      L.n = (int32_t)p.cols[0][b].second;
      int64_t lc = o.leaf_rank_cap ? o.leaf_rank_cap : 1024;
      L.rcap = (int32_t)std::min<int64_t>(std::min<int64_t>(L.m, L.n), lc);
      L.tape_iters = std::min(L.m, L.n);
      L.stream_id = ((int64_t)a << 12) | b;
      L.u_off = uo;
      L.v_off = vo;
      L.tape_off = to;
      L.taped_off = tdo;
      uo += (int64_t)L.m * L.rcap;
      vo += (int64_t)L.rcap * L.n;
      to += (int64_t)L.tape_iters * rec;
      tdo += (int64_t)L.tape_iters * 2;
      p.mmax = std::max(p.mmax, L.m);
      p.nmax = std::max(p.nmax, L.n);
      p.rcap_max = std::max(p.rcap_max, L.rcap);
    }

  // ---- BACA cluster size: enough CTAs to cover the SMs, shared memory within budget
  int c = o.cluster;
  if (c == 0) {
    c = 1;
    while (c < 8 && (int64_t)p.nleaves * c < 2 * sms && (p.mmax + c * 2 - 1) / (c * 2) >= 16) c *= 2;
  }
  while (baca_smem(p.esz, (p.mmax + c - 1) / c, (p.nmax + c - 1) / c, p.d) > 200 * 1024 && c < 16) c *= 2;
  p.baca_cluster = c;
  p.mr_max = (p.mmax + c - 1) / c;
  p.nc_max = (p.nmax + c - 1) / c;
  p.baca_smem = baca_smem(p.esz, p.mr_max, p.nc_max, p.d);
  if (p.baca_smem > 227 * 1024) { err = "leaf too large for shared memory even with 16-CTA clusters"; return false; }
  {
    // resident clusters are bounded by SMs x CTAs per SM / c
    size_t per_sm = std::min<size_t>(8, std::max<size_t>(1, (228 * 1024) / (p.baca_smem + 1024)));
    p.max_clusters_scratch = (int)std::max<int64_t>(1, std::min<int64_t>(p.nleaves, (int64_t)sms * per_sm / c));
  }
  p.cscr_stride = (int64_t)p.mmax * p.d;
  p.rscr_stride = (int64_t)p.d * p.nmax;
  p.gscr_stride = (int64_t)2 * c * p.rcap_max * p.d;

  // ---- stores and stages
  const int64_t cap = p.rank_cap;
  // full store levels 0..L-1 (level L goes to the user), half store levels 1..L
  struct BlockPlan { std::vector<BlockRef> refs; };
  std::vector<BlockPlan> full(p.L + 1), half(p.L + 1);
  size_t full_u = 0, full_s = 0, full_v = 0, half_u = 0, half_s = 0, half_v = 0;
  for (int l = 0; l < p.L; ++l) {
    int64_t u = 0, s = 0, v = 0;
    const int nr = (int)p.rows[l].size(), ncn = (int)p.cols[l].size();
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < ncn; ++b) {
        BlockRef r{};
        r.m = (int32_t)p.rows[l][a].second;
        r.n = (int32_t)p.cols[l][b].second;
        r.u_off = u; r.s_off = s; r.v_off = v;
        r.ldu = r.m; r.ldv = r.n;
        r.rank_slot = a * ncn + b;
        u += r.m * cap; s += cap; v += cap * r.n;
        full[l].refs.push_back(r);
      }
    full_u = std::max<size_t>(full_u, u); full_s = std::max<size_t>(full_s, s); full_v = std::max<size_t>(full_v, v);
  }
  for (int l = 1; l <= p.L; ++l) {
    int64_t u = 0, s = 0, v = 0;
    const int nr = (int)p.rows[l - 1].size(), ncn = (int)p.cols[l].size();
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < ncn; ++b) {
        BlockRef r{};
        r.m = (int32_t)p.rows[l - 1][a].second;
        r.n = (int32_t)p.cols[l][b].second;
        r.u_off = u; r.s_off = s; r.v_off = v;
        r.ldu = r.m; r.ldv = r.n;
        r.rank_slot = a * ncn + b;
        u += r.m * cap; s += cap; v += cap * r.n;
        half[l].refs.push_back(r);
      }
    half_u = std::max<size_t>(half_u, u); half_s = std::max<size_t>(half_s, s); half_v = std::max<size_t>(half_v, v);
  }

  // tasks, grouped into chunks whose scratch (QR operands, cores) fits the budget;
  // scratch offsets are local to a chunk, chunks of a stage run one after another
  p.task_storage.clear();
  p.stages.clear();
  size_t qr_elems = 0, tau_elems = 0, core_elems = 0, ord_elems = 0;
  const size_t budget = (size_t)8 << 30;  // bytes of chunk scratch
  auto add_stage = [&](std::vector<SvdTask>& all, int kind, int in_store, int in_level, int out_store, int out_level) {
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
      st.in_store = in_store; st.in_level = in_level;
      st.out_store = out_store; st.out_level = out_level;
      p.task_storage.push_back(ch);
      p.stages.push_back(st);
    }
  };
  {
    std::vector<SvdTask> ts(p.nleaves);
    for (int i = 0; i < p.nleaves; ++i) {
      SvdTask& t = ts[i];
      std::memset(&t, 0, sizeof(t));
      t.kind = TASK_LEAF;
      t.kcap = leaves[i].rcap;
      t.in1 = i;
      t.a_off = leaves[i].u_off;
      t.a_in_baca = 1;
      t.rows_a = leaves[i].m;
      t.lda = leaves[i].m;
      t.rows_b = leaves[i].n;
      t.src_v_off = leaves[i].v_off;
      t.out = i;
    }
    add_stage(ts, TASK_LEAF, -1, 0, p.L == 0 ? 2 : 0, 0);
  }
  for (int l = 1; l <= p.L; ++l) {
    const int64_t kc = std::min<int64_t>(2 * cap, 2 * mn);
    {  // horizontal: row nodes at level l-1, column nodes at level l
      const int nr = (int)p.rows[l - 1].size(), ncn = (int)p.cols[l].size(), ncp = (int)p.cols[l - 1].size();
      std::vector<SvdTask> ts;
      for (int a = 0; a < nr; ++a)
        for (int b = 0; b < ncn; ++b) {
          SvdTask t;
          std::memset(&t, 0, sizeof(t));
          t.kind = TASK_HORIZ;
          t.kcap = (int32_t)kc;
          t.in1 = a * ncp + 2 * b;
          t.in2 = a * ncp + 2 * b + 1;
          t.rows_a = (int32_t)p.rows[l - 1][a].second;
          t.lda = t.rows_a;
          t.out = a * ncn + b;
          t.m1 = (int32_t)p.cols[l - 1][2 * b].second;
          ts.push_back(t);
        }
      add_stage(ts, TASK_HORIZ, 0, l - 1, 1, l);
    }
    {  // vertical: row and column nodes at level l; children in the half store
      const int nr = (int)p.rows[l].size(), ncn = (int)p.cols[l].size();
      std::vector<SvdTask> ts;
      for (int a = 0; a < nr; ++a)
        for (int b = 0; b < ncn; ++b) {
          SvdTask t;
          std::memset(&t, 0, sizeof(t));
          t.kind = TASK_VERT;
          t.kcap = (int32_t)kc;
          t.in1 = (2 * a) * ncn + b;
          t.in2 = (2 * a + 1) * ncn + b;
          t.rows_a = (int32_t)p.cols[l][b].second;
          t.lda = t.rows_a;
          t.out = a * ncn + b;
          t.m1 = (int32_t)p.rows[l - 1][2 * a].second;
          ts.push_back(t);
        }
      add_stage(ts, TASK_VERT, 1, l, l == p.L ? 2 : 0, l);
    }
  }
  for (size_t i = 0; i < p.stages.size(); ++i) p.stages[i].tasks_h = &p.task_storage[i];

  // ---- descriptor staging (host-written) and device-written tables
  std::vector<char>& D = p.desc;
  D.clear();
  auto put = [&](const void* src, size_t bytes) {
    size_t off = D.size();
    D.resize(align_up(off + bytes));
    if (bytes) std::memcpy(D.data() + off, src, bytes);
    return off;
  };
  p.leafdesc_off = put(leaves.data(), leaves.size() * sizeof(LeafDesc));
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
        QJob b{};
        b.task = i;
        b.which = 1;
        b.to_v = 1;
        aj.push_back(b);
      }
    }
    st.nqr = (int)qj.size();
    st.nq = (int)aj.size();
    st.qrjobs_off = put(qj.data(), qj.size() * sizeof(QrJob));
    st.qjobs_off = put(aj.data(), aj.size() * sizeof(QJob));
  }
  p.full_lv.assign(p.L + 1, StoreLevel());
  p.half_lv.assign(p.L + 1, StoreLevel());
  for (int l = 0; l < p.L; ++l) {
    p.full_lv[l].nblocks = (int)full[l].refs.size();
    p.full_lv[l].refs_off = put(full[l].refs.data(), full[l].refs.size() * sizeof(BlockRef));
  }
  for (int l = 1; l <= p.L; ++l) {
    p.half_lv[l].nblocks = (int)half[l].refs.size();
    p.half_lv[l].refs_off = put(half[l].refs.data(), half[l].refs.size() * sizeof(BlockRef));
  }
  {
    BlockRef u{};
    u.m = (int32_t)g.m;
    u.n = (int32_t)g.n;
    u.ldu = g.m;
    u.ldv = g.n;
    p.user_ref_off = put(&u, sizeof(u));
    p.user_lv.nblocks = 1;
    p.user_lv.refs_off = p.user_ref_off;
  }

  Layout Lo;
  p.status = Lo.take(64);
  p.queue = Lo.take(64);
  p.desc_region = Lo.take(D.size());
  Region leafout = Lo.take((size_t)p.nleaves * sizeof(LeafOut));
  p.leafout_off = leafout.off;
  // device-written rank tables and task dims
  for (int l = 0; l < p.L; ++l) p.full_lv[l].rank_off = Lo.take((size_t)p.full_lv[l].nblocks * 4).off;
  for (int l = 1; l <= p.L; ++l) p.half_lv[l].rank_off = Lo.take((size_t)p.half_lv[l].nblocks * 4).off;
  p.user_lv.rank_off = Lo.take(4).off;
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
  p.total = Lo.cur;
  return true;
}

void bind_user_result(Plan& p, const hbaca_result& r) {
  BlockRef u{};
  u.m = (int32_t)p.m;
  u.n = (int32_t)p.n;
  u.ldu = r.ldu;
  u.ldv = r.ldv;
  u.rank_slot = 0;
  std::memcpy(p.desc.data() + p.user_ref_off, &u, sizeof(u));
}

}  // namespace hbaca
