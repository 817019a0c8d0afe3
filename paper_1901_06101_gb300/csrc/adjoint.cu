// y = U diag(S) V X (hbaca_apply) and its reverse pass with frozen pivots
// (hbaca_apply_backward): real double precision, Gaussian entry generator.
//
// The backward reads the sizes the forward left in its workspace (ranks,
// kept/stored triplet counts, leaf pivot records; one device-to-host copy),
// lays out its own workspace, and runs a fixed list of batched launches:
//   1. for the merge tree from the root down, the adjoint of every truncated
//      SVD node (all nodes of a stage in one batch of launches);
//   2. for every leaf, the adjoint of its BACA factors, then the reverse BACA
//      iterations (Alg. 2 run backwards, with R_k regenerated from the factors
//      rather than stored);
//   3. the adjoint of the entry generator: dL/dx, dL/dy, dL/dh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint_kernels.cuh"
#include "hbaca.h"
#include "plan.h"
#include "run.h"
#include "types.h"

namespace hbaca {
namespace {

constexpr size_t kTapeMarkOffset = 16;
constexpr unsigned char kTapeMarkByte = 0x5A;

enum StepKind { ST_GEMM, ST_COPY, ST_GAP, ST_GENROWS, ST_LEAFSTEP, ST_ADJCOLS, ST_ADJROWS };

struct Step {
  int kind;
  size_t off;      // task array offset in the blob
  int ntasks;
  int64_t grid;    // CTAs (GEMM) or chunks (others)
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t cur = 0;
  size_t take(size_t bytes) {
    const size_t o = cur;
    cur = align256(cur + std::max<size_t>(bytes, 1));
    return o;
  }
};

// Launch list with task arrays in one host blob (copied to the device once).
struct Program {
  std::vector<char> blob;
  std::vector<Step> steps;
  int sms = 152;
  template <class T>
  size_t put(const std::vector<T>& v) {
    const size_t off = blob.size();
    blob.resize(align256(off + v.size() * sizeof(T)));
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
  void gemm(std::vector<GemmTask> ts) {
    std::vector<GemmTask> keep;
    int64_t tiles = 0;
    for (GemmTask& t : ts) {
      if (t.M <= 0 || t.N <= 0 || (t.K <= 0 && !t.beta0)) continue;
      t.tm = (t.M + kGemmTile - 1) / kGemmTile;
      t.tn = (t.N + kGemmTile - 1) / kGemmTile;
      tiles += (int64_t)t.tm * t.tn;
      keep.push_back(t);
    }
    if (keep.empty()) return;
    int64_t first = 0;
    for (GemmTask& t : keep) {
      int ks = 1;
      if (!t.beta0 && t.K > 256) {
        const int64_t want = std::max<int64_t>(1, (3 * (int64_t)sms) / std::max<int64_t>(1, tiles));
        ks = (int)std::min<int64_t>(want, t.K / 128);
        ks = std::max(ks, 1);
      }
      t.ksplit = ks;
      t.first = first;
      first += (int64_t)t.tm * t.tn * ks;
    }
    steps.push_back(Step{ST_GEMM, put(keep), (int)keep.size(), first});
  }
  void copy(const std::vector<CopyTask>& ts) {
    std::vector<CopyTask> keep;
    for (const CopyTask& t : ts)
      if (t.rows > 0 && t.cols > 0) keep.push_back(t);
    if (!keep.empty()) steps.push_back(Step{ST_COPY, put(keep), (int)keep.size(), 32});
  }
  template <class T>
  void add(int kind, const std::vector<T>& ts, int64_t grid) {
    if (!ts.empty()) steps.push_back(Step{kind, put(ts), (int)ts.size(), grid});
  }
};

GemmTask gemm_task(int M, int N, int K, double alpha, const double* A, int64_t a_ri, int64_t a_ki, const double* B,
                   int64_t b_ki, int64_t b_cj, double* C, int64_t c_ri, int64_t c_cj, bool beta0) {
  GemmTask t;
  std::memset(&t, 0, sizeof(t));
  t.M = M;
  t.N = N;
  t.K = K;
  t.ksplit = 1;
  t.beta0 = beta0 ? 1 : 0;
  t.alpha = alpha;
  t.A = A;
  t.a_ri = a_ri;
  t.a_ki = a_ki;
  t.B = B;
  t.b_ki = b_ki;
  t.b_cj = b_cj;
  t.C = C;
  t.c_ri = c_ri;
  t.c_cj = c_cj;
  return t;
}

CopyTask copy_task(int64_t rows, int64_t cols, const double* src, int64_t s_ri, int64_t s_cj, double* dst,
                   int64_t d_ri, int64_t d_cj) {
  return CopyTask{rows, cols, src, s_ri, s_cj, dst, d_ri, d_cj};
}

cudaError_t run_program(const Program& pg, char* dev_blob, cudaStream_t st, int& launches) {
  cudaError_t e = cudaSuccess;
  if (!pg.blob.empty()) e = cudaMemcpyAsync(dev_blob, pg.blob.data(), pg.blob.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(leafstep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafStepSmem);
  if (e != cudaSuccess) return e;
  for (const Step& s : pg.steps) {
    const void* tp = dev_blob + s.off;
    switch (s.kind) {
      case ST_GEMM:
        gemm_kernel<<<(unsigned)s.grid, kGemmThreads, 0, st>>>(reinterpret_cast<const GemmTask*>(tp), s.ntasks);
        break;
      case ST_COPY:
        copy_kernel<<<dim3((unsigned)s.grid, s.ntasks), 256, 0, st>>>(reinterpret_cast<const CopyTask*>(tp));
        break;
      case ST_GAP:
        gap_kernel<<<dim3((unsigned)s.grid, s.ntasks), 256, 0, st>>>(reinterpret_cast<const GapTask*>(tp));
        break;
      case ST_GENROWS:
        genrows_kernel<<<dim3((unsigned)s.grid, s.ntasks), 256, 0, st>>>(reinterpret_cast<const GenRowsTask*>(tp));
        break;
      case ST_LEAFSTEP:
        leafstep_kernel<<<s.ntasks, 32, kLeafStepSmem, st>>>(reinterpret_cast<const LeafStepTask*>(tp));
        break;
      case ST_ADJCOLS:
        genadj_cols_kernel<<<dim3((unsigned)s.grid, s.ntasks), kAdjThreads, 0, st>>>(
            reinterpret_cast<const GenAdjTask*>(tp));
        break;
      case ST_ADJROWS:
        genadj_rows_kernel<<<dim3((unsigned)s.grid, s.ntasks), kAdjThreads, 0, st>>>(
            reinterpret_cast<const GenAdjTask*>(tp));
        break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++launches;
  }
  return cudaSuccess;
}

bool check_real_gauss(const hbaca_gen* gen, std::string& err) {
  if (!gen) { err = "gen is NULL"; return false; }
  if (gen->dtype != HBACA_F64) { err = "the backward pass is available for real (F64) matrices"; return false; }
  if (gen->kind != HBACA_GEN_GAUSSIAN) { err = "the backward pass is available for the GAUSSIAN generator"; return false; }
  if (gen->dim < 1 || gen->dim > kMaxDim) { err = "Gaussian point dimension must be 1..4 for the backward pass"; return false; }
  if (!(gen->h > 0.0)) { err = "Gaussian h must be > 0"; return false; }
  return true;
}

// Sizes the forward left in its workspace.
struct TapeSizes {
  std::vector<int32_t> ranks;
  std::vector<LeafOut> leafout;
  std::vector<std::vector<TaskDims>> dims;
  std::vector<std::vector<int32_t>> tape;  // per leaf: iters x (4 + 3d)
};

bool read_sizes(const Plan& p, const char* ws, cudaStream_t st, TapeSizes& ts, std::string& err) {
  // the mark first (the status region is at the start of every layout): a
  // workspace of an untaped call is smaller than this plan and must not be
  // read further
  unsigned char mark[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(mark, ws + p.status.off + kTapeMarkOffset, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("reading the tape mark: ") + cudaGetErrorString(e); return false; }
  for (int i = 0; i < 4; ++i)
    if (mark[i] != kTapeMarkByte) {
      err = "the workspace holds no tape: compress with HBACA_FLAG_TAPE first";
      return false;
    }
  ts.ranks.assign(p.nslots, 0);
  ts.leafout.resize(p.nleaves);
  e = cudaMemcpyAsync(ts.ranks.data(), ws + p.ranks_off, (size_t)p.nslots * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ts.leafout.data(), ws + p.leafout_off, (size_t)p.nleaves * sizeof(LeafOut), cudaMemcpyDeviceToHost, st);
  ts.dims.resize(p.stages.size());
  for (size_t si = 0; si < p.stages.size() && e == cudaSuccess; ++si) {
    ts.dims[si].resize(p.stages[si].ntasks);
    e = cudaMemcpyAsync(ts.dims[si].data(), ws + p.stages[si].dims_off, ts.dims[si].size() * sizeof(TaskDims),
                        cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("reading the tape sizes: ") + cudaGetErrorString(e); return false; }
  const int rec = 4 + 3 * p.d;
  ts.tape.resize(p.nleaves);
  const LeafDesc* leaves = reinterpret_cast<const LeafDesc*>(p.desc.data() + p.leafdesc_off);
  for (int l = 0; l < p.nleaves && e == cudaSuccess; ++l) {
    const int it = std::min(ts.leafout[l].iters, leaves[l].tape_iters);
    ts.tape[l].assign((size_t)std::max(it, 0) * rec, 0);
    if (it > 0)
      e = cudaMemcpyAsync(ts.tape[l].data(), ws + p.tape_int.off + leaves[l].tape_off * 4, (size_t)it * rec * 4,
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("reading the pivot records: ") + cudaGetErrorString(e); return false; }
  return true;
}

// Incoming adjoint of a node: Abar = P Q^T, P (rows x rho, ld ldp), Q (cols x rho, ld ldq).
struct Adj {
  const double* P = nullptr;
  int64_t ldp = 0;
  const double* Q = nullptr;
  int64_t ldq = 0;
  int rho = 0;
  bool set = false;
};

struct NodeRec {
  int stage, task, kind;
  int ref;                   // producing task's output ref
  int s, nout;
  int64_t m, n;
  const double* U;           // m x nout, col-major (ld m)
  const double* S;
  const double* V;           // nout x n, row-major (ld n)
  Adj in;
  // buffers (offsets in the backward workspace)
  size_t A1, B1, AB, GB, GC, E1, E2, Pp, Qp;
};

struct LeafRec {
  int leaf, block;
  int64_t m, n, row0, col0;
  int rB;                    // BACA rank
  const double* UB;          // m x rB (ld m)
  const double* VB;          // rB x n (ld n)
  Adj in;
  size_t Ubar, Vbar, Acols, Arows, Rk, Zbar, Z, G1, G2, slotcol, rowidx;
  int nrow;                  // rows of Arows
  struct It { int dI, dk, r0, rowoff; const int32_t* I; const int32_t* J; const int32_t* jbar; };
  std::vector<It> its;       // iterations with dk > 0, in forward order
  std::vector<int32_t> rowidx_h;
};

// Everything the backward needs, laid out and programmed.
struct Backward {
  Layout lay;
  std::vector<NodeRec> nodes;
  std::vector<LeafRec> leaves;
  Program pg;
  size_t zero_bytes = 0;  // buffers [0, zero_bytes) of the backward workspace start at zero
  size_t blob_off = 0;    // the launch program's task arrays
  size_t total = 0;
};

// Caller arrays of one block of a backward call (device pointers).
struct BlockArgs {
  const double* X;
  int64_t ldx;
  const double* dY;
  int64_t lddy;
  const double* U;  // the forward's result
  int64_t ldu;
  const double* S;
  const double* V;
  int64_t ldv;
  int rank;
  double* dX;       // may be null
  int64_t lddx;
  double* d_x;      // gradient outputs (may be null)
  double* d_y;
  double* d_h;
};

struct BwdArgs {
  int64_t nrhs;
  std::vector<BlockArgs> blk;
};

// Lay out the backward workspace at base address `bws` and program every
// launch.  With a placeholder base the result gives the exact size.
bool build_backward(const Plan& p, const char* ws, const TapeSizes& ts, const BwdArgs& ar, char* bws, Backward& bw,
                    std::string& err) {
  const int64_t nrhs = ar.nrhs;
  const BlockRef* refs = reinterpret_cast<const BlockRef*>(p.desc.data() + p.refs_off);
  const LeafDesc* leafd = reinterpret_cast<const LeafDesc*>(p.desc.data() + p.leafdesc_off);
  const double* fullU = reinterpret_cast<const double*>(ws + p.full_u.off);
  const double* fullS = reinterpret_cast<const double*>(ws + p.full_s.off);
  const double* fullV = reinterpret_cast<const double*>(ws + p.full_v.off);
  const double* halfU = reinterpret_cast<const double*>(ws + p.half_u.off);
  const double* halfS = reinterpret_cast<const double*>(ws + p.half_s.off);
  const double* halfV = reinterpret_cast<const double*>(ws + p.half_v.off);
  Layout& L = bw.lay;
  auto D = [&](size_t off) { return reinterpret_cast<double*>(bws + off); };
  auto I32 = [&](size_t off) { return reinterpret_cast<int32_t*>(bws + off); };

  // ---- nodes (one per task of every stage), producer map
  std::vector<int> node_of_ref(p.nrefs, -1);
  for (size_t si = 0; si < p.stages.size(); ++si) {
    const Stage& sg = p.stages[si];
    for (int ti = 0; ti < sg.ntasks; ++ti) {
      const SvdTask& t = (*sg.tasks_h)[ti];
      NodeRec nd;
      std::memset(&nd, 0, sizeof(nd));
      nd.stage = (int)si;
      nd.task = ti;
      nd.kind = t.kind;
      nd.ref = t.out;
      const BlockRef& r = refs[t.out];
      if (r.full_slot < 0) { err = "workspace layout has no tape"; return false; }
      nd.s = ts.ranks[r.rank_slot];
      nd.nout = ts.ranks[r.full_slot];
      nd.m = r.m;
      nd.n = r.n;
      const bool half = sg.out_store == 1;
      nd.U = (half ? halfU : fullU) + r.u_off;
      nd.S = (half ? halfS : fullS) + r.s_off;
      nd.V = (half ? halfV : fullV) + r.v_off;
      if (nd.s < 0 || nd.nout < nd.s || nd.nout > r.store_cap) { err = "inconsistent tape sizes"; return false; }
      node_of_ref[t.out] = (int)bw.nodes.size();
      bw.nodes.push_back(nd);
    }
  }
  // ---- the root of every block receives (dY, X)
  for (int b = 0; b < p.nblocks; ++b) {
    const int rn = node_of_ref[p.root_tape_first + b];
    if (rn < 0) { err = "no root node"; return false; }
    Adj a;
    a.P = ar.blk[b].dY;
    a.ldp = ar.blk[b].lddy;
    a.Q = ar.blk[b].X;
    a.ldq = ar.blk[b].ldx;
    a.rho = (int)nrhs;
    a.set = true;
    bw.nodes[rn].in = a;
  }
  // ---- leaves
  const int rec = 4 + 3 * p.d;
  bw.leaves.resize(p.nleaves);
  for (int l = 0; l < p.nleaves; ++l) {
    LeafRec& lr = bw.leaves[l];
    const LeafDesc& Ld = leafd[l];
    lr.leaf = l;
    lr.block = Ld.block;
    lr.m = Ld.m;
    lr.n = Ld.n;
    lr.row0 = Ld.row0;
    lr.col0 = Ld.col0;
    lr.rB = ts.leafout[l].rank;
    lr.UB = reinterpret_cast<const double*>(ws + p.uar.off) + Ld.u_off;
    lr.VB = reinterpret_cast<const double*>(ws + p.var.off) + Ld.v_off;
    const int32_t* tape_dev = reinterpret_cast<const int32_t*>(ws + p.tape_int.off) + Ld.tape_off;
    int r0 = 0, rowoff = 0;
    const int nit = (int)(ts.tape[l].size() / rec);
    for (int it = 0; it < nit; ++it) {
      const int32_t* rr = ts.tape[l].data() + (size_t)it * rec;
      const int dI = rr[0], dk = rr[2];
      if (dk <= 0) continue;
      if (dI > kMaxD || dk > kMaxD || dk > dI) { err = "pivot record out of range"; return false; }
      LeafRec::It x;
      x.dI = dI;
      x.dk = dk;
      x.r0 = r0;
      x.rowoff = rowoff;
      x.I = tape_dev + (size_t)it * rec + 4;
      x.J = tape_dev + (size_t)it * rec + 4 + p.d;
      x.jbar = tape_dev + (size_t)it * rec + 4 + 2 * p.d;
      for (int i = 0; i < dI; ++i) lr.rowidx_h.push_back(rr[4 + i]);
      lr.its.push_back(x);
      r0 += dk;
      rowoff += dI;
    }
    if (r0 != lr.rB) { err = "leaf rank does not match its pivot record"; return false; }
    lr.nrow = rowoff;
  }

  // ---- buffers
  const int64_t rho_max = std::max<int64_t>(2 * p.rank_cap_max, nrhs);  // rho = nrhs (root) or 2 s_parent
  for (NodeRec& nd : bw.nodes) {
    const int64_t rho = rho_max;
    nd.A1 = L.take((size_t)nd.nout * rho * 8);
    nd.B1 = L.take((size_t)nd.nout * rho * 8);
    nd.AB = L.take((size_t)nd.s * nd.s * 8);
    nd.GB = L.take((size_t)nd.s * (nd.nout - nd.s) * 8);
    nd.GC = L.take((size_t)nd.s * (nd.nout - nd.s) * 8);
    nd.E1 = L.take((size_t)nd.s * (nd.nout - nd.s) * 8);
    nd.E2 = L.take((size_t)nd.s * (nd.nout - nd.s) * 8);
    nd.Pp = L.take((size_t)nd.m * 2 * nd.s * 8);
    nd.Qp = L.take((size_t)nd.n * 2 * nd.s * 8);
  }
  for (LeafRec& lr : bw.leaves) {
    const int64_t rB = std::max(lr.rB, 1);
    const int64_t rho = 2 * p.rank_cap_max;  // a leaf receives rho = 2 s of its re-compression node
    lr.Ubar = L.take((size_t)lr.m * rB * 8);
    lr.Vbar = L.take((size_t)rB * lr.n * 8);
    lr.Acols = L.take((size_t)lr.m * rB * 8);
    lr.Arows = L.take((size_t)std::max(lr.nrow, 1) * lr.n * 8);
    lr.Rk = L.take((size_t)kMaxD * lr.n * 8);
    lr.Zbar = L.take((size_t)kMaxD * kMaxD * 8);
    lr.Z = L.take((size_t)kMaxD * kMaxD * 8);
    lr.G1 = L.take((size_t)rB * rho * 8);
    lr.G2 = L.take((size_t)rB * rho * 8);
    lr.slotcol = L.take((size_t)rB * 4);
    lr.rowidx = L.take((size_t)std::max(lr.nrow, 1) * 4);
  }
  std::vector<size_t> t2(p.nblocks);  // U^T dY for dX, per block
  for (int b = 0; b < p.nblocks; ++b) t2[b] = L.take((size_t)std::max(ar.blk[b].rank, 1) * nrhs * 8);
  bw.zero_bytes = L.cur;
  // the entry generator of a block and where its gradients go
  auto gauss_of = [&](int b) {
    GaussAdj G;
    const hbaca_gen& g = p.gens[b];
    G.x = g.x;
    G.y = g.y;
    G.dim = g.dim;
    G.h = g.h;
    G.c = -1.0 / (2.0 * g.h * g.h);
    G.dx = ar.blk[b].d_x;
    G.dy = ar.blk[b].d_y;
    G.dh = ar.blk[b].d_h;
    return G;
  };

  Program& pg = bw.pg;

  // ---- merge tree, stages from last to first
  for (int si = (int)p.stages.size() - 1; si >= 0; --si) {
    std::vector<int> ids;
    for (size_t k = 0; k < bw.nodes.size(); ++k)
      if (bw.nodes[k].stage == si && bw.nodes[k].in.set && bw.nodes[k].in.rho > 0 && bw.nodes[k].s > 0)
        ids.push_back((int)k);
    std::vector<GemmTask> g1, g2, g3;
    std::vector<GapTask> gaps;
    std::vector<CopyTask> cps;
    for (int k : ids) {
      NodeRec& nd = bw.nodes[k];
      const Adj& a = nd.in;
      const int s = nd.s, nout = nd.nout, nd_ = nout - s, rho = a.rho;
      const int64_t m = nd.m, n = nd.n;
      // A1 = U_all^T P (nout x rho), B1 = V_all Q (nout x rho)
      g1.push_back(gemm_task(nout, rho, (int)m, 1.0, nd.U, m, 1, a.P, 1, a.ldp, D(nd.A1), 1, nout, false));
      g1.push_back(gemm_task(nout, rho, (int)n, 1.0, nd.V, n, 1, a.Q, 1, a.ldq, D(nd.B1), 1, nout, false));
      // AB = a b^T (s x s); GB = a vd^T (s x nd); GC = ud b^T (nd x s)
      g2.push_back(gemm_task(s, s, rho, 1.0, D(nd.A1), 1, nout, D(nd.B1), nout, 1, D(nd.AB), 1, s, false));
      if (nd_ > 0) {
        g2.push_back(gemm_task(s, nd_, rho, 1.0, D(nd.A1), 1, nout, D(nd.B1) + s, nout, 1, D(nd.GB), 1, s, false));
        g2.push_back(gemm_task(nd_, s, rho, 1.0, D(nd.A1) + s, 1, nout, D(nd.B1), nout, 1, D(nd.GC), 1, nd_, false));
        gaps.push_back(GapTask{s, nd_, nd.S, D(nd.GB), D(nd.GC), D(nd.E1), D(nd.E2)});
      }
      double* Pp = D(nd.Pp);  // m x 2s: [U_r, Psi]
      double* Qp = D(nd.Qp);  // n x 2s: [Phi, V_r^T]
      cps.push_back(copy_task(m, s, nd.U, 1, m, Pp, 1, m));
      cps.push_back(copy_task(n, s, nd.V, 1, n, Qp + (size_t)s * n, 1, n));
      // Phi = Q a^T (+ V_d^T E1^T);  Psi = P b^T - U_r (a b^T) (+ U_d E2)
      g3.push_back(gemm_task((int)n, s, rho, 1.0, a.Q, 1, a.ldq, D(nd.A1), nout, 1, Qp, 1, n, false));
      g3.push_back(gemm_task((int)m, s, rho, 1.0, a.P, 1, a.ldp, D(nd.B1), nout, 1, Pp + (size_t)s * m, 1, m, false));
      g3.push_back(gemm_task((int)m, s, s, -1.0, nd.U, 1, m, D(nd.AB), 1, s, Pp + (size_t)s * m, 1, m, false));
      if (nd_ > 0) {
        g3.push_back(gemm_task((int)n, s, nd_, 1.0, nd.V + (size_t)s * n, 1, n, D(nd.E1), s, 1, Qp, 1, n, false));
        g3.push_back(gemm_task((int)m, s, nd_, 1.0, nd.U + (size_t)s * m, 1, m, D(nd.E2), 1, nd_, Pp + (size_t)s * m, 1, m,
                               false));
      }
      // children
      const SvdTask& t = (*p.stages[si].tasks_h)[nd.task];
      Adj c1, c2;
      c1.rho = c2.rho = 2 * s;
      c1.set = c2.set = true;
      if (nd.kind == TASK_LEAF) {
        c1.P = Pp; c1.ldp = m; c1.Q = Qp; c1.ldq = n;
        bw.leaves[t.in1].in = c1;
      } else if (nd.kind == TASK_HORIZ) {
        c1.P = Pp; c1.ldp = m; c1.Q = Qp; c1.ldq = n;
        c2 = c1;
        c2.Q = Qp + t.m1;
        const int n1 = node_of_ref[t.in1], n2 = node_of_ref[t.in2];
        if (n1 < 0 || n2 < 0) { err = "merge child without producer"; return false; }
        bw.nodes[n1].in = c1;
        bw.nodes[n2].in = c2;
      } else {
        c1.P = Pp; c1.ldp = m; c1.Q = Qp; c1.ldq = n;
        c2 = c1;
        c2.P = Pp + t.m1;
        const int n1 = node_of_ref[t.in1], n2 = node_of_ref[t.in2];
        if (n1 < 0 || n2 < 0) { err = "merge child without producer"; return false; }
        bw.nodes[n1].in = c1;
        bw.nodes[n2].in = c2;
      }
    }
    pg.gemm(g1);
    pg.gemm(g2);
    pg.add(ST_GAP, gaps, 32);
    pg.copy(cps);
    pg.gemm(g3);
  }

  // ---- leaves: Ubar = P (Q^T V_B^T), Vbar = (U_B^T P) Q^T
  {
    std::vector<GemmTask> a, b;
    for (LeafRec& lr : bw.leaves) {
      if (!lr.in.set || lr.in.rho <= 0 || lr.rB <= 0) continue;
      const int rho = lr.in.rho, rB = lr.rB;
      const int64_t m = lr.m, n = lr.n;
      a.push_back(gemm_task(rB, rho, (int)n, 1.0, lr.VB, n, 1, lr.in.Q, 1, lr.in.ldq, D(lr.G1), 1, rB, false));
      a.push_back(gemm_task(rB, rho, (int)m, 1.0, lr.UB, m, 1, lr.in.P, 1, lr.in.ldp, D(lr.G2), 1, rB, false));
      b.push_back(gemm_task((int)m, rB, rho, 1.0, lr.in.P, 1, lr.in.ldp, D(lr.G1), rB, 1, D(lr.Ubar), 1, m, false));
      b.push_back(gemm_task(rB, (int)n, rho, 1.0, D(lr.G2), 1, rB, lr.in.Q, lr.in.ldq, 1, D(lr.Vbar), n, 1, false));
    }
    pg.gemm(a);
    pg.gemm(b);
  }

  // ---- reverse BACA iterations
  {
    // row index arrays: copied into the workspace through the blob
    std::vector<int32_t> allrows;
    std::vector<std::pair<size_t, size_t>> spans;  // (blob element offset, leaf)
    int kmax = 0;
    for (LeafRec& lr : bw.leaves) kmax = std::max<int>(kmax, (int)lr.its.size());
    for (int step = 0; step < kmax; ++step) {
      std::vector<GemmTask> gR, gZ, gRbar, gUp;
      std::vector<GenRowsTask> gen;
      std::vector<CopyTask> cp;
      std::vector<LeafStepTask> ls;
      for (LeafRec& lr : bw.leaves) {
        if (!lr.in.set || lr.in.rho <= 0) continue;
        const int K = (int)lr.its.size();
        const int k = K - 1 - step;
        if (k < 0) continue;
        const LeafRec::It& it = lr.its[k];
        const int64_t m = lr.m, n = lr.n;
        const int r0 = it.r0, dI = it.dI, dk = it.dk;
        double* Rk = D(lr.Rk);
        double* Ub = D(lr.Ubar);
        double* Vb = D(lr.Vbar);
        double* Ac = D(lr.Acols);
        double* Ar = D(lr.Arows) + (size_t)it.rowoff * n;
        // R_k = A(I_k, :) - U_B(I_k, 0:r0) V_B(0:r0, :)
        GemmTask t = gemm_task(dI, (int)n, r0, -1.0, lr.UB, 1, m, lr.VB, n, 1, Rk, n, 1, true);
        t.amap = it.I;
        gR.push_back(t);
        gen.push_back(GenRowsTask{dI, (int)n, it.I, Rk, lr.row0, lr.col0, gauss_of(lr.block)});
        // Zbar = Vbar(r0:r0+dk, :) R_k^T  (dk x dI)
        gZ.push_back(gemm_task(dk, dI, (int)n, 1.0, Vb + (size_t)r0 * n, n, 1, Rk, 1, n, D(lr.Zbar), 1, dk, true));
        // Acols(:, r0:r0+dk) = Ubar(:, r0:r0+dk), then the LRID step adds Wbar at rows I_k
        cp.push_back(copy_task(m, dk, Ub + (size_t)r0 * m, 1, m, Ac + (size_t)r0 * m, 1, m));
        LeafStepTask st;
        std::memset(&st, 0, sizeof(st));
        st.dI = dI;
        st.dk = dk;
        st.n = (int)n;
        st.m = (int)m;
        st.r0 = r0;
        st.R = Rk;
        st.I = it.I;
        st.J = it.J;
        st.jbar = it.jbar;
        st.Zbar = D(lr.Zbar);
        st.Z = D(lr.Z);
        st.Acols = Ac;
        st.slotcol = I32(lr.slotcol);
        ls.push_back(st);
        // Rbar_k = Z^T Vbar(r0:r0+dk, :)  (dI x n) into its rows of Arows
        gRbar.push_back(gemm_task(dI, (int)n, dk, 1.0, D(lr.Z), dk, 1, Vb + (size_t)r0 * n, n, 1, Ar, n, 1, true));
        if (r0 > 0) {
          const int32_t* jc = I32(lr.slotcol) + r0;
          // Ubar(:, 0:r0) -= Cbar V_B(0:r0, jcols)^T
          GemmTask u1 = gemm_task((int)m, r0, dk, -1.0, Ac + (size_t)r0 * m, 1, m, lr.VB, 1, n, Ub, 1, m, false);
          u1.bkmap = jc;
          gUp.push_back(u1);
          // Vbar(0:r0, jcols) -= U_B(:, 0:r0)^T Cbar
          GemmTask u2 = gemm_task(r0, dk, (int)m, -1.0, lr.UB, m, 1, Ac + (size_t)r0 * m, 1, m, Vb, n, 1, false);
          u2.cmap_c = jc;
          gUp.push_back(u2);
          // Ubar(I_k, 0:r0) -= Rbar_k V_B(0:r0, :)^T
          GemmTask u3 = gemm_task(dI, r0, (int)n, -1.0, Ar, n, 1, lr.VB, 1, n, Ub, 1, m, false);
          u3.cmap_r = it.I;
          gUp.push_back(u3);
          // Vbar(0:r0, :) -= U_B(I_k, 0:r0)^T Rbar_k
          GemmTask u4 = gemm_task(r0, (int)n, dI, -1.0, lr.UB, m, 1, Ar, n, 1, Vb, n, 1, false);
          u4.akmap = it.I;
          gUp.push_back(u4);
        }
      }
      pg.gemm(gR);
      pg.add(ST_GENROWS, gen, 16);
      pg.gemm(gZ);
      pg.copy(cp);
      pg.add(ST_LEAFSTEP, ls, 0);
      pg.gemm(gRbar);
      pg.gemm(gUp);
    }
  }

  // ---- generator adjoint
  {
    std::vector<GenAdjTask> tc, tr;
    int64_t gm = 1, gn = 1;
    for (LeafRec& lr : bw.leaves) {
      if (!lr.in.set || lr.in.rho <= 0 || lr.rB <= 0) continue;
      GenAdjTask t;
      std::memset(&t, 0, sizeof(t));
      t.m = (int)lr.m;
      t.n = (int)lr.n;
      t.nslot = lr.rB;
      t.nrow = lr.nrow;
      t.row0 = lr.row0;
      t.col0 = lr.col0;
      t.Acols = D(lr.Acols);
      t.slotcol = I32(lr.slotcol);
      t.Arows = D(lr.Arows);
      t.rowidx = I32(lr.rowidx);
      t.G = gauss_of(lr.block);
      tc.push_back(t);
      tr.push_back(t);
      gm = std::max<int64_t>(gm, (lr.m + kAdjThreads - 1) / kAdjThreads);
      gn = std::max<int64_t>(gn, (lr.n + kAdjThreads - 1) / kAdjThreads);
    }
    pg.add(ST_ADJCOLS, tc, gm);
    pg.add(ST_ADJROWS, tr, gn);
  }

  // ---- dX = V^T diag(S) (U^T dY), per block
  {
    std::vector<GemmTask> a, b2;
    for (int b = 0; b < p.nblocks; ++b) {
      const BlockArgs& ba = ar.blk[b];
      if (!ba.dX || ba.rank <= 0) continue;
      const int r = ba.rank;
      const int64_t m = p.gens[b].m, n = p.gens[b].n;
      a.push_back(gemm_task(r, (int)nrhs, (int)m, 1.0, ba.U, ba.ldu, 1, ba.dY, 1, ba.lddy, D(t2[b]), 1, r, false));
      GemmTask t = gemm_task((int)n, (int)nrhs, r, 1.0, ba.V, 1, ba.ldv, D(t2[b]), 1, r, ba.dX, 1, ba.lddx, false);
      t.akscale = ba.S;
      b2.push_back(t);
    }
    pg.gemm(a);
    pg.gemm(b2);
  }
  bw.blob_off = align256(bw.zero_bytes);
  bw.total = bw.blob_off + align256(pg.blob.size());
  return true;
}

}  // namespace
}  // namespace hbaca

using namespace hbaca;

namespace {

// Plan of the forward and the sizes it left in its workspace.
bool load_forward(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts, const void* workspace, int64_t nrhs,
                  void* stream, Plan& p, TapeSizes& ts, int& sms, std::string& err) {
  if (!gens || nblocks < 1) { err = "gens is NULL or nblocks < 1"; return false; }
  for (int b = 0; b < nblocks; ++b)
    if (!check_real_gauss(gens + b, err)) return false;
  if (!opts || !workspace) { err = "opts or workspace is NULL"; return false; }
  if (nrhs < 1) { err = "nrhs must be >= 1"; return false; }
  if (!(opts->flags & HBACA_FLAG_TAPE)) { err = "opts must carry HBACA_FLAG_TAPE (the flags of the forward call)"; return false; }
  int dev = 0;
  sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  if (!make_plan(gens, nblocks, *opts, sms, p, err)) return false;
  return read_sizes(p, reinterpret_cast<const char*>(workspace), reinterpret_cast<cudaStream_t>(stream), ts, err);
}

int root_rank(const Plan& p, const TapeSizes& ts, int b) {
  const BlockRef* refs = reinterpret_cast<const BlockRef*>(p.desc.data() + p.refs_off);
  return ts.ranks[refs[p.root_tape_first + b].rank_slot];
}

// Arguments with placeholder pointers: the backward's layout does not depend
// on the caller's arrays, only on the sizes.
BwdArgs placeholder_args(const Plan& p, const TapeSizes& ts, int64_t nrhs) {
  static const double kDummy[1] = {0.0};
  BwdArgs ar;
  ar.nrhs = nrhs;
  for (int b = 0; b < p.nblocks; ++b) {
    const int64_t m = p.gens[b].m, n = p.gens[b].n;
    ar.blk.push_back(BlockArgs{kDummy, n, kDummy, m, kDummy, m, kDummy, kDummy, n, root_rank(p, ts, b),
                               const_cast<double*>(kDummy), n, nullptr, nullptr, nullptr});
  }
  return ar;
}

size_t backward_size(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts, const void* workspace,
                     int64_t nrhs, void* stream) {
  Plan p;
  TapeSizes ts;
  int sms = 152;
  std::string err;
  if (!load_forward(nblocks, gens, opts, workspace, nrhs, stream, p, ts, sms, err)) {
    record_error(HBACA_INVALID_ARG, err);
    return 0;
  }
  const BwdArgs ar = placeholder_args(p, ts, nrhs);
  Backward bw;
  bw.pg.sms = sms;
  char* base = reinterpret_cast<char*>(static_cast<uintptr_t>(4096));
  if (!build_backward(p, reinterpret_cast<const char*>(workspace), ts, ar, base, bw, err)) {
    record_error(HBACA_INVALID_ARG, err);
    return 0;
  }
  record_error(HBACA_OK, "");
  return bw.total;
}

// The reverse pass over the blocks of one forward call; `ar.blk` holds the
// caller's arrays of every block.
hbaca_status backward(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts, const void* workspace,
                      BwdArgs& ar, void* bwd_workspace, size_t bwd_bytes, void* stream) {
  if (!bwd_workspace) return record_error(HBACA_INVALID_ARG, "NULL backward workspace");
  if (reinterpret_cast<uintptr_t>(bwd_workspace) & 255u)
    return record_error(HBACA_WORKSPACE, "backward workspace must be 256-byte aligned");
  Plan p;
  TapeSizes ts;
  int sms = 152;
  std::string err;
  if (!load_forward(nblocks, gens, opts, workspace, ar.nrhs, stream, p, ts, sms, err))
    return record_error(HBACA_INVALID_ARG, err);
  for (int b = 0; b < nblocks; ++b) {
    const BlockArgs& ba = ar.blk[b];
    if (!ba.X || !ba.dY) return record_error(HBACA_INVALID_ARG, "NULL X or dY");
    if (ba.ldx < gens[b].n || ba.lddy < gens[b].m || (ba.dX && ba.lddx < gens[b].n))
      return record_error(HBACA_INVALID_ARG, "leading dimensions too small");
    if (ba.rank != root_rank(p, ts, b))
      return record_error(HBACA_INVALID_ARG, "result rank differs from the tape's root rank");
  }
  char* bws = reinterpret_cast<char*>(bwd_workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Backward bw;
  bw.pg.sms = sms;
  if (!build_backward(p, reinterpret_cast<const char*>(workspace), ts, ar, bws, bw, err))
    return record_error(HBACA_INVALID_ARG, err);
  if (bw.total > bwd_bytes)
    return record_error(HBACA_WORKSPACE, "backward workspace too small (hbaca_backward_workspace_size gives the size)");
  // zero the buffers and the outputs, upload the row indices, run
  cudaError_t e = cudaMemsetAsync(bws, 0, bw.zero_bytes, st);
  for (int b = 0; b < nblocks && e == cudaSuccess; ++b) {
    const BlockArgs& ba = ar.blk[b];
    if (ba.dX)
      for (int64_t c = 0; c < ar.nrhs && e == cudaSuccess; ++c)
        e = cudaMemsetAsync(ba.dX + c * ba.lddx, 0, (size_t)gens[b].n * 8, st);
    if (e == cudaSuccess && ba.d_x) e = cudaMemsetAsync(ba.d_x, 0, (size_t)gens[b].m * gens[b].dim * 8, st);
    if (e == cudaSuccess && ba.d_y) e = cudaMemsetAsync(ba.d_y, 0, (size_t)gens[b].n * gens[b].dim * 8, st);
    if (e == cudaSuccess && ba.d_h) e = cudaMemsetAsync(ba.d_h, 0, 8, st);
  }
  for (size_t l = 0; l < bw.leaves.size() && e == cudaSuccess; ++l) {
    const LeafRec& lr = bw.leaves[l];
    if (!lr.rowidx_h.empty())
      e = cudaMemcpyAsync(bws + lr.rowidx, lr.rowidx_h.data(), lr.rowidx_h.size() * 4, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return record_error(HBACA_CUDA, std::string("backward set-up: ") + cudaGetErrorString(e));
  int launches = 0;
  e = run_program(bw.pg, bws + bw.blob_off, st, launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return record_error(HBACA_CUDA, std::string("backward: ") + cudaGetErrorString(e));
  return record_error(HBACA_OK, "");
}

BlockArgs block_args(const hbaca_result& r, const void* X, int64_t ldx, const void* dY, int64_t lddy, void* dX,
                     int64_t lddx, double* d_x, double* d_y, double* d_h) {
  return BlockArgs{reinterpret_cast<const double*>(X), ldx, reinterpret_cast<const double*>(dY), lddy,
                   reinterpret_cast<const double*>(r.U), r.ldu, r.S, reinterpret_cast<const double*>(r.V), r.ldv,
                   (int)r.rank, reinterpret_cast<double*>(dX), lddx, d_x, d_y, d_h};
}

}  // namespace

extern "C" {

size_t hbaca_apply_workspace_size(int64_t rank_cap, int64_t nrhs) {
  if (rank_cap < 1 || nrhs < 1) return 0;
  return align256((size_t)rank_cap * nrhs * 8) + 4096;
}

hbaca_status hbaca_apply(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_result* res, const void* X, int64_t nrhs,
                         int64_t ldx, void* Y, int64_t ldy, void* workspace, void* stream) {
  if (!ctx || !gen || !res || !X || !Y || !workspace) return record_error(HBACA_INVALID_ARG, "NULL argument");
  if (gen->dtype != HBACA_F64) return record_error(HBACA_INVALID_ARG, "hbaca_apply is available for real (F64) results");
  if (nrhs < 1 || ldx < gen->n || ldy < gen->m) return record_error(HBACA_INVALID_ARG, "need nrhs >= 1, ldx >= n, ldy >= m");
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return record_error(HBACA_WORKSPACE, "workspace must be 256-byte aligned");
  const int r = res->rank;
  if (r < 0) return record_error(HBACA_INVALID_ARG, "result has no host rank (compressed with HBACA_FLAG_ASYNC)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  const size_t tbytes = align256((size_t)std::max(r, 1) * nrhs * 8);
  double* Tm = reinterpret_cast<double*>(ws);
  Program pg;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&pg.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int64_t m = gen->m, n = gen->n;
  const double* U = reinterpret_cast<const double*>(res->U);
  const double* V = reinterpret_cast<const double*>(res->V);
  double* Yd = reinterpret_cast<double*>(Y);
  pg.copy({copy_task(m, nrhs, nullptr, 0, 0, Yd, 1, ldy), copy_task(std::max(r, 1), nrhs, nullptr, 0, 0, Tm, 1, std::max(r, 1))});
  if (r > 0) {
    // T = V X (r x nrhs); Y = U diag(S) T
    pg.gemm({gemm_task(r, (int)nrhs, (int)n, 1.0, V, res->ldv, 1, reinterpret_cast<const double*>(X), 1, ldx, Tm, 1, r,
                       false)});
    GemmTask t = gemm_task((int)m, (int)nrhs, r, 1.0, U, 1, res->ldu, Tm, 1, r, Yd, 1, ldy, false);
    t.akscale = res->S;
    pg.gemm({t});
  }
  if (tbytes + pg.blob.size() > hbaca_apply_workspace_size(std::max(r, 1), nrhs))
    return record_error(HBACA_WORKSPACE, "apply workspace too small");
  int launches = 0;
  cudaError_t e = run_program(pg, ws + tbytes, st, launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return record_error(HBACA_CUDA, std::string("apply: ") + cudaGetErrorString(e));
  return record_error(HBACA_OK, "");
}

size_t hbaca_backward_workspace_size(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace, int64_t nrhs,
                                     void* stream) {
  return backward_size(1, gen, opts, workspace, nrhs, stream);
}

size_t hbaca_backward_workspace_size_batched(int32_t nblocks, const hbaca_gen* gens, const hbaca_opts* opts,
                                             const void* workspace, int64_t nrhs, void* stream) {
  return backward_size(nblocks, gens, opts, workspace, nrhs, stream);
}

hbaca_status hbaca_apply_backward(hbaca_ctx* ctx, const hbaca_gen* gen, const hbaca_opts* opts, const hbaca_result* res,
                                  const void* workspace, const void* X, int64_t nrhs, int64_t ldx, const void* dY,
                                  int64_t lddy, double* d_h, double* d_x, double* d_y, void* dX, int64_t lddx,
                                  void* bwd_workspace, size_t bwd_bytes, void* stream) {
  if (!ctx || !res || !X || !dY || !gen) return record_error(HBACA_INVALID_ARG, "NULL argument");
  BwdArgs ar;
  ar.nrhs = nrhs;
  ar.blk.push_back(block_args(*res, X, ldx, dY, lddy, dX, lddx, d_x, d_y, d_h));
  return backward(1, gen, opts, workspace, ar, bwd_workspace, bwd_bytes, stream);
}

hbaca_status hbaca_apply_backward_batched(hbaca_ctx* ctx, int32_t nblocks, const hbaca_gen* gens,
                                          const hbaca_opts* opts, const hbaca_result* results, const void* workspace,
                                          const void* const* X, int64_t nrhs, const void* const* dY, double* d_h,
                                          double* const* d_x, double* const* d_y, void* const* dX,
                                          void* bwd_workspace, size_t bwd_bytes, void* stream) {
  if (!ctx || !gens || !results || !X || !dY || nblocks < 1) return record_error(HBACA_INVALID_ARG, "NULL argument");
  BwdArgs ar;
  ar.nrhs = nrhs;
  for (int b = 0; b < nblocks; ++b)
    ar.blk.push_back(block_args(results[b], X[b], gens[b].n, dY[b], gens[b].m, dX ? dX[b] : nullptr, gens[b].n,
                                d_x ? d_x[b] : nullptr, d_y ? d_y[b] : nullptr, d_h ? d_h + b : nullptr));
  return backward(nblocks, gens, opts, workspace, ar, bwd_workspace, bwd_bytes, stream);
}

int64_t hbaca_debug_backward_json(const hbaca_gen* gen, const hbaca_opts* opts, const void* workspace, int64_t nrhs,
                                  char* buf, int64_t len, void* stream) {
  Plan p;
  TapeSizes ts;
  int sms = 152;
  std::string err;
  if (!load_forward(1, gen, opts, workspace, nrhs, stream, p, ts, sms, err)) {
    record_error(HBACA_INVALID_ARG, err);
    return -1;
  }
  const BwdArgs ar = placeholder_args(p, ts, nrhs);
  Backward bw;
  bw.pg.sms = sms;
  char* base = reinterpret_cast<char*>(static_cast<uintptr_t>(4096));
  if (!build_backward(p, reinterpret_cast<const char*>(workspace), ts, ar, base, bw, err)) {
    record_error(HBACA_INVALID_ARG, err);
    return -1;
  }
  const LeafDesc* leafd = reinterpret_cast<const LeafDesc*>(p.desc.data() + p.leafdesc_off);
  std::string j = "{\"total\": " + std::to_string(bw.total) + ", \"leaves\": [";
  for (size_t l = 0; l < bw.leaves.size(); ++l) {
    const LeafRec& r = bw.leaves[l];
    j += "{\"Ubar\": " + std::to_string(r.Ubar) + ", \"Vbar\": " + std::to_string(r.Vbar) +
         ", \"Acols\": " + std::to_string(r.Acols) + ", \"Arows\": " + std::to_string(r.Arows) +
         ", \"slotcol\": " + std::to_string(r.slotcol) + ", \"rowidx\": " + std::to_string(r.rowidx) +
         ", \"rB\": " + std::to_string(r.rB) + ", \"nrow\": " + std::to_string(r.nrow) +
         ", \"m\": " + std::to_string(r.m) + ", \"n\": " + std::to_string(r.n) +
         ", \"u_off\": " + std::to_string(p.uar.off + leafd[l].u_off * 8) +
         ", \"v_off\": " + std::to_string(p.var.off + leafd[l].v_off * 8) + "}";
    if (l + 1 < bw.leaves.size()) j += ", ";
  }
  j += "], \"nodes\": [";
  for (size_t k = 0; k < bw.nodes.size(); ++k) {
    const NodeRec& r = bw.nodes[k];
    j += "{\"stage\": " + std::to_string(r.stage) + ", \"task\": " + std::to_string(r.task) +
         ", \"kind\": " + std::to_string(r.kind) + ", \"s\": " + std::to_string(r.s) +
         ", \"nout\": " + std::to_string(r.nout) + ", \"m\": " + std::to_string(r.m) +
         ", \"n\": " + std::to_string(r.n) + ", \"rho\": " + std::to_string(r.in.rho) +
         ", \"A1\": " + std::to_string(r.A1) + ", \"B1\": " + std::to_string(r.B1) +
         ", \"Pp\": " + std::to_string(r.Pp) + ", \"Qp\": " + std::to_string(r.Qp) +
         ", \"U\": " + std::to_string(reinterpret_cast<const char*>(r.U) - reinterpret_cast<const char*>(workspace)) +
         ", \"V\": " + std::to_string(reinterpret_cast<const char*>(r.V) - reinterpret_cast<const char*>(workspace)) +
         ", \"S\": " + std::to_string(reinterpret_cast<const char*>(r.S) - reinterpret_cast<const char*>(workspace)) + "}";
    if (k + 1 < bw.nodes.size()) j += ", ";
  }
  j += "]}";
  if (buf && len > 0) {
    const size_t c = std::min<size_t>((size_t)len - 1, j.size());
    std::memcpy(buf, j.data(), c);
    buf[c] = 0;
  }
  record_error(HBACA_OK, "");
  return (int64_t)j.size() + 1;
}

}  // extern "C"
