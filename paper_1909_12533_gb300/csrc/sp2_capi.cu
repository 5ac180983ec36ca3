// C ABI (include/sp2.h) and the host side of the SP2ACC expansion:
//   Section 4 Step 1 -- schedule (p_i, alpha_i, n_min, n_max, tau_i), Algorithm 1;
//   Section 4 Step 2 -- Algorithm 2 (loop, stop test);
//   Section 4 Step 3 -- homo/lumo estimates.
// Every matrix operation is a kernel of this library on the caller's stream; the
// host only sees scalars (tile counts, e_i, t_i, lambda bounds).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>
#include <mutex>

#include "sp2_internal.h"

using namespace sp2;

namespace sp2 {
thread_local long long g_launches = 0;
}

namespace {

constexpr double C_STOP = 6.8872;  // Algorithm 2

// ------------------------------------------------------------------ schedule
// Reading of Step 1 (the companion paper's Algorithm 4 is not reproduced in
// the paper): eigenvalue images are tracked as intervals [vlo, vhi] (virtual,
// near 0) and [olo, ohi] (occupied, near 1).  p = 1 (x^2) iff the virtual
// interval is farther from 0 than the occupied one is from 1; while
// acceleration is on, alpha folds the improved interval symmetrically about
// the vertex of the polynomial (scale-and-fold); it switches off for good once
// both distances are <= delta_acc.  Truncation with ||E||_2 <= tau widens both
// intervals by tau (Weyl).  n_max: steps until both slack-free intervals are
// within 2^-52 of {0, 1}.
double poly_scalar(int p, double a, double x) {
  if (p == 1) {
    const double y = (1.0 - a) + a * x;
    return y * y;
  }
  const double ax = a * x;
  return (2.0 * a) * x - ax * ax;
}

void image(int p, double a, double& lo, double& hi) {
  const double f1 = poly_scalar(p, a, lo), f2 = poly_scalar(p, a, hi);
  double mn = std::min(f1, f2), mx = std::max(f1, f2);
  const double vertex = (p == 1) ? (a - 1.0) / a : 1.0 / a;
  if (lo <= vertex && vertex <= hi) {
    const double fv = poly_scalar(p, a, vertex);
    mn = std::min(mn, fv);
    mx = std::max(mx, fv);
  }
  lo = mn;
  hi = mx;
}

void choose(double vlo, double vhi, double olo, double ohi, bool& acc, double delta_acc, int& p, double& alpha) {
  const double d0 = std::max(vhi, -vlo);
  const double d1 = std::max(1.0 - olo, ohi - 1.0);
  p = d0 > d1 ? 1 : 0;
  if (acc && std::max(d0, d1) > delta_acc) {
    alpha = (p == 1) ? 2.0 / ((2.0 - vlo) - vhi) : 2.0 / (olo + ohi);
    alpha = std::max(alpha, 1.0);
    return;
  }
  acc = false;
  alpha = 1.0;
}

struct Schedule {
  double lmin = 0, lmax = 0;
  std::vector<int> p;
  std::vector<double> alpha, tau, vhi, olo;
  int n_min = 1, n_max = 0;
};

Schedule make_schedule(double lmin, double lmax, double homo_ub, double lumo_lb, double tau, double gamma,
                       bool accelerate, double delta_acc, int n_cap) {
  Schedule s;
  s.lmin = lmin;
  s.lmax = lmax;
  const double w = lmax - lmin;
  const double v0 = (lmax - lumo_lb) / w, o0 = (lmax - homo_ub) / w;
  double vlo = 0.0, vhi = v0, olo = o0, ohi = 1.0;
  bool acc = accelerate;
  int n_max = n_cap;
  for (int i = 1; i <= n_cap; ++i) {
    int p;
    double a;
    choose(vlo, vhi, olo, ohi, acc, delta_acc, p, a);
    image(p, a, vlo, vhi);
    image(p, a, olo, ohi);
    if (std::max(std::max(vhi, -vlo), std::max(1.0 - olo, ohi - 1.0)) < std::ldexp(1.0, -52)) {
      n_max = i;
      break;
    }
  }
  s.n_max = n_max;
  auto tau_of = [&](double vh, double ol) {
    if (!(gamma > 0.0)) return tau;
    const double g = gamma / (double)(n_max + 1);
    return g * (ol - vh) / (1.0 + g);
  };
  vlo = 0.0; vhi = v0; olo = o0; ohi = 1.0;
  double t0 = tau_of(vhi, olo);
  s.tau.push_back(t0);
  vlo -= t0; vhi += t0; olo -= t0; ohi += t0;
  s.p.push_back(-1);
  s.alpha.push_back(NAN);
  s.vhi.push_back(vhi);
  s.olo.push_back(olo);
  acc = accelerate;
  s.n_min = accelerate ? n_max + 1 : 1;
  for (int i = 1; i <= n_max; ++i) {
    int p;
    double a;
    const bool was = acc;
    choose(vlo, vhi, olo, ohi, acc, delta_acc, p, a);
    if (was && !acc) s.n_min = i;
    s.p.push_back(p);
    s.alpha.push_back(a);
    image(p, a, vlo, vhi);
    image(p, a, olo, ohi);
    const double ti = tau_of(vhi, olo);
    s.tau.push_back(ti);
    vlo -= ti; vhi += ti; olo -= ti; ohi += ti;
    s.vhi.push_back(vhi);
    s.olo.push_back(olo);
  }
  return s;
}

// Trace-correcting expansion (Section 1): no bounds, so no schedule ahead of
// time -- p_i is chosen from trace(X~_{i-1}) during the run, alpha_i = 1,
// n_min = 1, n_max = the cap, tau_i = tau.
Schedule make_schedule_trace(double lmin, double lmax, double tau, int n_cap) {
  Schedule s;
  s.lmin = lmin;
  s.lmax = lmax;
  s.n_max = n_cap;
  s.n_min = 1;
  s.p.assign(n_cap + 1, -1);
  s.alpha.assign(n_cap + 1, 1.0);
  s.alpha[0] = NAN;
  s.tau.assign(n_cap + 1, tau);
  s.vhi.assign(n_cap + 1, NAN);
  s.olo.assign(n_cap + 1, NAN);
  return s;
}

void coeffs(int p, double a, double& c0, double& c1, double& c2) {
  if (p == 1) {
    c0 = (1.0 - a) * (1.0 - a);
    c1 = 2.0 * a * (1.0 - a);
    c2 = a * a;
  } else {
    c0 = 0.0;
    c1 = 2.0 * a;
    c2 = -(a * a);
  }
}

// ------------------------------------------------------------------ Step 3
// Reading of Step 3 (the interior-eigenvalue paper's Algorithm 3 is not
// reproduced in the paper): every eigenvalue image x of X~_j adds r = x - x^2 to
// t_j and r^2 to e_j^2.  A step with x^2 (p_j = 1) squares r on the virtual side
// and about doubles it on the occupied side, so right after it the occupied side
// carries e_j and t_j; after 2x - x^2 the virtual side does.  On that side the
// largest r is estimated by e_j^2 / t_j, x = (1 +/- sqrt(1 - 4r)) / 2 next to the
// gap, then x is pulled back through f_j..f_1 (gap-side branch) and X_0's map.
// Per side the largest j with e_j > 100 f, t_j > 10 f, 10 f < r < 1/4 is used,
// f = tau_j + sqrt(N) 2^-52.  Through scale-and-fold steps the gap-side branch
// is an assumption (the fold maps two preimages onto one image).
double pull_back(const Schedule& s, int j, double x) {
  for (int i = j; i >= 1; --i) {
    const int p = s.p[i];
    const double a = s.alpha[i];
    const double y = std::min(std::max(x, 0.0), 1.0);
    if (p == 1) x = (std::sqrt(y) + a - 1.0) / a;
    else x = (1.0 - std::sqrt(1.0 - y)) / a;
  }
  return s.lmax - x * (s.lmax - s.lmin);
}

void estimates(const Schedule& s, const std::vector<double>& e, const std::vector<double>& t, int64_t n,
               double& homo, double& lumo, int& have) {
  homo = lumo = NAN;
  have = 0;
  bool hf = false, lf = false;
  for (int j = (int)t.size() - 1; j >= 1; --j) {
    if (j >= (int)s.p.size()) continue;
    const double f = s.tau[std::min<size_t>(j, s.tau.size() - 1)] + std::sqrt((double)n) * std::ldexp(1.0, -52);
    if (!(e[j] > 100.0 * f && t[j] > 10.0 * f)) continue;
    const double r = e[j] * e[j] / t[j];
    if (!(10.0 * f < r && r < 0.25)) continue;
    if (s.p[j] == 1 && !hf) {
      homo = pull_back(s, j, (1.0 + std::sqrt(1.0 - 4.0 * r)) / 2.0);
      hf = true;
    } else if (s.p[j] == 0 && !lf) {
      lumo = pull_back(s, j, (1.0 - std::sqrt(1.0 - 4.0 * r)) / 2.0);
      lf = true;
    }
    if (hf && lf) break;
  }
  have = (hf ? 1 : 0) | (lf ? 2 : 0);
}

// ------------------------------------------------------------------ memory
// One stream-ordered memory pool per device, kept for the life of the process
// with no release threshold: a context created after another was destroyed
// takes its memory from the pool instead of the driver.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

// Page-locked host scratch of a context (step scalars, counts): blocks of the
// process are kept on a free list, so creating a context costs no page-locked
// allocation after the first.
struct HostBlock {
  StepScalars sc;
  int32_t cnt[4];
  double d2[2];
};
std::mutex g_host_mu;
std::vector<HostBlock*> g_host_free;

HostBlock* take_host_block() {
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    if (!g_host_free.empty()) {
      HostBlock* b = g_host_free.back();
      g_host_free.pop_back();
      return b;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, sizeof(HostBlock)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<HostBlock*>(p);
}

void give_host_block(HostBlock* b) {
  if (!b) return;
  std::lock_guard<std::mutex> lk(g_host_mu);
  g_host_free.push_back(b);
}

struct Alloc {
  sp2_allocator a{};
  bool custom = false;
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (custom) return a.alloc(bytes, a.user);
    void* p = nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p) {
    if (!p) return;
    if (custom) {
      cudaStreamSynchronize(st);  // the caller's free is not stream-ordered
      a.free(p, a.user);
    } else {
      cudaFreeAsync(p, st);
    }
  }
};

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  template <class T> T* as() const { return static_cast<T*>(p); }
};

struct Fail {
  int code;
};

// Device buffers of one tensor-core operand: super-row bitmaps, per-word
// record counts and offsets, record index words, headers and slices.
struct OpBufs {
  Buf sbits, cnt, spos, index, head, data;
};

// Per-iteration record for the adjoint: the kept tiles of X~_j and, every
// ckpt_every steps, their FP64 values (contiguous, index order).
struct Rec {
  Buf brow, bcol, rowptr, val;
  int64_t nnzb = 0;
  bool has_val = false;
};

}  // namespace

struct sp2_ctx {
  Alloc al;
  cudaStream_t st = nullptr;
  sp2_params prm{};
  int64_t n = 0, nocc = 0;
  int nb = 0, words = 0;
  double homo_ub = 0, lumo_lb = 0, tau = 0;
  Schedule sch;
  std::vector<Buf*> bufs;
  // F (kept for the adjoint) and X~ (current iterate, values in pool[cur])
  TileSet F, X, out;
  Buf f_brow, f_bcol, f_slot, f_rowptr, f_pool;
  Buf x_brow, x_bcol, x_slot, x_rowptr;      // index set 0 of X~
  Buf y_brow, y_bcol, y_slot, y_rowptr;      // index set 1 (the next X~ while the stop test is pending)
  int xset = 0;
  int tail_from = 0;   // first iteration of the FP64 tail (0: none yet)
  int selftest_pending = 0;   // error-path self-test still to run (1 timeout, 2 range)
  Buf o_brow, o_bcol, o_slot, o_rowptr, o_bits;
  Buf pool[2];
  int cur = 0;
  FullPattern fp;
  Buf fp_bits, fp_rowptr, fp_col, fp_ref, counts;
  Buf p_e2, p_trS, p_trX, p_n2, p_kt, keep, scanbuf, scantmp, twork, rowlo, rowhi;
  Buf dsc, dcnt, d2;
  OpBufs opx, opy;   // tensor-core operands (the adjoint uses both)
  Buf sflag, spos, slist, errflag, scount, tcscratch, redwork;
  // adjoint
  std::vector<Rec> recs;
  std::vector<Buf> seg;
  Buf ident, fpB_bits, fpB_rowptr, fpB_col, fpB_ref, gpool[2], w_brow, w_bcol, w_rowptr, w_pool, dF;
  Buf amax, trbuf, dsq, rsq;
  Buf gflag, gpos, gkeep, u_brow, u_bcol, u_slot;   // general storage: upper sub-index
  FullPattern fpB;
  double backward_ms = 0.0;
  HostBlock* hb = nullptr;
  StepScalars* h_sc = nullptr;
  int32_t* h_cnt = nullptr;
  double* h_d2 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs0 = nullptr, evs1 = nullptr;
  // outputs
  Buf d_brow, d_bcol, d_val;
  int64_t d_nnzb = 0;
  bool ran = false, have_D = false;
  sp2_stats stats{};
  std::string last_error;

  sp2_ctx() {
    Buf* all[] = {&f_brow, &f_bcol, &f_slot, &f_rowptr, &f_pool, &x_brow, &x_bcol, &x_slot, &x_rowptr,
                  &y_brow, &y_bcol, &y_slot, &y_rowptr,
                  &o_brow, &o_bcol, &o_slot, &o_rowptr, &o_bits, &pool[0], &pool[1], &fp_bits, &fp_rowptr,
                  &fp_col, &fp_ref, &counts, &p_e2, &p_trS, &p_trX, &p_n2, &p_kt, &keep, &scanbuf, &scantmp,
                  &twork, &rowlo, &rowhi, &dsc, &dcnt, &d2, &d_brow, &d_bcol, &d_val, &opx.sbits,
                  &opx.cnt, &opx.spos, &opx.index, &opx.head, &opx.data, &opy.sbits, &opy.cnt, &opy.spos,
                  &opy.index, &opy.head, &opy.data, &sflag, &spos, &slist, &errflag, &scount, &tcscratch, &redwork, &ident, &fpB_bits, &fpB_rowptr, &fpB_col,
                  &fpB_ref, &gpool[0], &gpool[1], &w_brow, &w_bcol, &w_rowptr, &w_pool, &dF, &amax, &trbuf, &dsq, &rsq, &gflag, &gpos, &gkeep,
                  &u_brow, &u_bcol, &u_slot};
    for (Buf* b : all) bufs.push_back(b);
  }

  void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      last_error = std::string(what) + ": " + cudaGetErrorString(e);
      throw Fail{SP2_ERR_CUDA};
    }
  }
  void ensure(Buf& b, size_t bytes) {
    if (b.cap >= bytes && b.p) return;
    al.put(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    b.p = al.get(want);
    if (!b.p) {
      last_error = "device allocation of " + std::to_string(want) + " bytes failed";
      throw Fail{SP2_ERR_OOM};
    }
    b.cap = want;
  }
  void sync() { ck(cudaStreamSynchronize(st), "stream sync"); }
};

namespace {

void set_tiles(TileSet& s, Buf& br, Buf& bc, Buf& sl, Buf& rp, int64_t nnzb) {
  s.nnzb = nnzb;
  s.brow = br.as<int32_t>();
  s.bcol = bc.as<int32_t>();
  s.slot = sl.as<int32_t>();
  s.rowptr = rp.as<int32_t>();
}

// Both-triangle pattern of a tile set (bitmap + neighbour lists).
void build_full(sp2_ctx* c, const TileSet& s, FullPattern& fp, Buf& bits, Buf& rowptr, Buf& col, Buf& ref) {
  c->ensure(bits, (size_t)c->nb * c->words * 4);
  c->ensure(rowptr, (size_t)(c->nb + 1) * 4);
  c->ensure(col, (size_t)std::max<int64_t>(2 * s.nnzb, 1) * 4);
  c->ensure(ref, (size_t)std::max<int64_t>(2 * s.nnzb, 1) * 4);
  c->ensure(c->counts, (size_t)(c->nb + 1) * 4);
  c->ensure(c->scantmp, scan_tmp_bytes(c->nb + 1) + scan_tmp_bytes(std::max<int64_t>(s.nnzb, c->nb)) + 4096);
  fp.words = c->words;
  fp.bits = bits.as<uint32_t>();
  fp.rowptr = rowptr.as<int32_t>();
  fp.col = col.as<int32_t>();
  fp.ref = ref.as<uint32_t>();
  fp.nnz = 2 * s.nnzb;
  c->ck(launch_bitmap(s, c->nb, fp, c->st), "bitmap");
  c->ck(launch_row_popc(fp.bits, c->nb, c->words, c->counts.as<int32_t>(), c->st), "row popc");
  c->ck(launch_scan_i32(c->counts.as<int32_t>(), fp.rowptr, c->nb, fp.rowptr + c->nb, c->scantmp.p, c->st),
        "scan");
  c->ck(launch_fill_full(s, c->nb, fp, c->st), "fill full");
}

void ensure_partials(sp2_ctx* c, int64_t nt) {
  const size_t d = (size_t)std::max<int64_t>(nt, 1) * 8, i4 = (size_t)std::max<int64_t>(nt, 1) * 4;
  c->ensure(c->p_e2, d);
  c->ensure(c->p_trS, d);
  c->ensure(c->p_trX, d);
  c->ensure(c->p_n2, d);
  c->ensure(c->p_kt, i4);
  c->ensure(c->keep, i4);
  c->ensure(c->scanbuf, i4);
}

Partials partials(sp2_ctx* c) {
  Partials p;
  p.e2 = c->p_e2.as<double>();
  p.trS = c->p_trS.as<double>();
  p.trX = c->p_trX.as<double>();
  p.n2 = c->p_n2.as<double>();
  p.ktiles = c->p_kt.as<int32_t>();
  return p;
}

int32_t read_count(sp2_ctx* c, const int32_t* dev) {
  c->ck(cudaMemcpyAsync(c->h_cnt, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st), "count d2h");
  c->sync();
  return *c->h_cnt;
}

// Truncate the tile set `in` (values indexed by slot, norms in n2[slot]) and
// compact its index into index set `set`; the kept-tile count is left in dcnt[0]
// (no host round trip).  Returns the target TileSet (nnzb not yet known).
// keep flags of the tiles of `in` under the context's truncation norm
void select_keep(sp2_ctx* c, const TileSet& in, const double* n2, double tau, int32_t* keep) {
  const int64_t part_tiles = std::max<int64_t>(1, c->prm.frobinf_part / TB);
  const int64_t nsb = (c->nb + part_tiles - 1) / part_tiles;
  if (c->prm.trunc == SP2_TRUNC_MIXED) {
    c->ensure(c->twork, mixed_work_bytes(std::max<int64_t>(in.nnzb, 1), (int)nsb));
    c->ck(mixed_select(in, n2, c->nb, tau, part_tiles, c->twork.p, keep, c->st), "mixed-norm truncation");
    return;
  }
  c->ensure(c->twork, trunc_work_bytes(std::max<int64_t>(in.nnzb, 1), c->nb, part_tiles));
  c->ck(launch_truncate(in, n2, c->nb, tau, c->prm.trunc, part_tiles, c->twork.p, keep, c->st), "truncate");
}

// Compact the tiles of `in` whose keep flag (c->keep) is set into index set
// `set`; the kept-tile count is left in dcnt[0] (no host round trip).
TileSet compact_into_set(sp2_ctx* c, const TileSet& in, int set) {
  const size_t cap = (size_t)std::max<int64_t>(in.nnzb, 1) * 4;
  Buf& br = set ? c->y_brow : c->x_brow;
  Buf& bc = set ? c->y_bcol : c->x_bcol;
  Buf& sl = set ? c->y_slot : c->x_slot;
  Buf& rp = set ? c->y_rowptr : c->x_rowptr;
  c->ensure(br, cap);
  c->ensure(bc, cap);
  c->ensure(sl, cap);
  c->ensure(rp, (size_t)(c->nb + 1) * 4);
  c->ensure(c->dcnt, 16);
  c->ensure(c->scanbuf, cap);
  c->ensure(c->scantmp, scan_tmp_bytes(in.nnzb) + 4096);
  TileSet t;
  set_tiles(t, br, bc, sl, rp, 0);
  c->ck(launch_compact(in, c->keep.as<int32_t>(), c->nb, t, c->dcnt.as<int32_t>(), c->scantmp.p,
                       c->scanbuf.as<int32_t>(), c->st),
        "compact");
  return t;
}

// Truncate the tile set `in` (values indexed by slot, norms in n2[slot]) and
// compact its index into index set `set`; the kept-tile count is left in dcnt[0]
// (no host round trip).  Returns the target TileSet (nnzb not yet known).
TileSet truncate_launch(sp2_ctx* c, const TileSet& in, const double* n2, double tau, int set) {
  // n2 may live in p_n2: only the flag buffers are (re)sized here
  c->ensure(c->keep, (size_t)std::max<int64_t>(in.nnzb, 1) * 4);
  select_keep(c, in, n2, tau, c->keep.as<int32_t>());
  return compact_into_set(c, in, set);
}

// General storage: the same selection as the symmetric storage, made on the
// upper tiles of `in` (all of its nb diagonal tiles are present, so there are
// (nnzb + nb) / 2 of them), then every lower tile follows its mirror.
TileSet truncate_launch_general(sp2_ctx* c, const TileSet& in, const double* n2, double tau, int set) {
  const int64_t nU = (in.nnzb + c->nb) / 2;
  const size_t cap = (size_t)std::max<int64_t>(in.nnzb, 1) * 4, capU = (size_t)std::max<int64_t>(nU, 1) * 4;
  c->ensure(c->gflag, cap);
  c->ensure(c->gpos, cap);
  c->ensure(c->gkeep, capU);
  c->ensure(c->u_brow, capU);
  c->ensure(c->u_bcol, capU);
  c->ensure(c->u_slot, capU);
  c->ensure(c->keep, cap);
  c->ensure(c->dcnt, 16);
  c->ensure(c->scantmp, scan_tmp_bytes(in.nnzb) + 4096);
  c->ck(launch_upper_flags(in, c->gflag.as<int32_t>(), c->st), "upper flags");
  TileSet U;
  U.nnzb = nU;
  U.brow = c->u_brow.as<int32_t>();
  U.bcol = c->u_bcol.as<int32_t>();
  U.slot = c->u_slot.as<int32_t>();
  U.rowptr = nullptr;
  c->ck(launch_compact(in, c->gflag.as<int32_t>(), c->nb, U, c->dcnt.as<int32_t>() + 1, c->scantmp.p,
                       c->gpos.as<int32_t>(), c->st),
        "upper tiles");
  select_keep(c, U, n2, tau, c->gkeep.as<int32_t>());
  c->ck(launch_general_keep(in, c->gpos.as<int32_t>(), c->gkeep.as<int32_t>(), c->keep.as<int32_t>(), c->st),
        "mirror keep");
  return compact_into_set(c, in, set);
}

// Make `t` (with its host-side count) the current X~ and build its row offsets.
void adopt_X(sp2_ctx* c, TileSet t, int64_t nnzb, int set) {
  t.nnzb = nnzb;
  c->X = t;
  c->xset = set;
  c->ck(launch_rowptr_from_brow(c->X.brow, c->X.nnzb, c->nb, c->X.rowptr, c->st), "rowptr");
}


void free_recs(sp2_ctx* c) {
  for (Rec& r : c->recs)
    for (Buf* b : {&r.brow, &r.bcol, &r.rowptr, &r.val}) {
      c->al.put(b->p);
      b->p = nullptr;
      b->cap = 0;
    }
  c->recs.clear();
  for (Buf& b : c->seg) c->al.put(b.p);
  c->seg.clear();
}

void ensure_ident(sp2_ctx* c, int64_t n) {
  if (c->ident.p && c->ident.cap >= (size_t)n * 4) return;
  c->ensure(c->ident, (size_t)std::max<int64_t>(n, 1) * 4);
  c->ck(launch_iota(c->ident.as<int32_t>(), (int64_t)(c->ident.cap / 4), c->st), "iota");
}

// General storage of X~_0: from the symmetric set c->X (values in pool[cur])
// to both triangles in index set 1 / pool[1 - cur], slots = tile index.
void expand_to_general(sp2_ctx* c) {
  build_full(c, c->X, c->fp, c->fp_bits, c->fp_rowptr, c->fp_col, c->fp_ref);
  const int64_t nG = read_count(c, c->fp.rowptr + c->nb);
  const size_t cap = (size_t)std::max<int64_t>(nG, 1) * 4;
  c->ensure(c->y_brow, cap);
  c->ensure(c->y_bcol, cap);
  c->ensure(c->y_slot, cap);
  c->ensure(c->y_rowptr, (size_t)(c->nb + 1) * 4);
  const int nxt = 1 - c->cur;
  c->ensure(c->pool[nxt], (size_t)std::max<int64_t>(nG, 1) * TE * 8);
  c->ck(launch_expand_general(c->fp, c->nb, c->pool[c->cur].as<double>(), c->y_brow.as<int32_t>(),
                              c->y_bcol.as<int32_t>(), c->pool[nxt].as<double>(), c->st),
        "expand");
  c->ck(launch_iota(c->y_slot.as<int32_t>(), nG, c->st), "slots");
  TileSet g;
  set_tiles(g, c->y_brow, c->y_bcol, c->y_slot, c->y_rowptr, 0);
  c->cur = nxt;
  adopt_X(c, g, nG, 1);
}

// Row (CSR) and column (CSC) views of the general X~ for the product: A reads
// row I's tiles (I, K) as stored, B reads column J's tiles (K, J) (REF_T:
// untransposed).  refs are pool slots (FP64 kernel) or tile indices (tensor
// path, whose operand records look the slots up).
void build_general(sp2_ctx* c, bool by_index) {
  const TileSet& X = c->X;
  c->ensure(c->fp_bits, (size_t)c->nb * c->words * 4);
  c->ck(launch_bits_general(X, c->nb, c->words, c->fp_bits.as<uint32_t>(), c->st), "bits");
  const int32_t* rslot = X.slot;
  if (by_index) {
    ensure_ident(c, X.nnzb);
    rslot = c->ident.as<int32_t>();
  }
  c->fp.words = c->words;
  c->fp.bits = c->fp_bits.as<uint32_t>();
  c->fp.rowptr = X.rowptr;
  c->fp.col = X.bcol;
  c->fp.ref = reinterpret_cast<uint32_t*>(const_cast<int32_t*>(rslot));
  c->fp.nnz = X.nnzb;
  c->ensure(c->fpB_ref, (size_t)std::max<int64_t>(X.nnzb, 1) * 4);
  c->ck(launch_csc_refs(X, by_index ? nullptr : X.slot, c->fpB_ref.as<uint32_t>(), c->st), "csc refs");
  c->fpB = c->fp;
  c->fpB.ref = c->fpB_ref.as<uint32_t>();
}

void record(sp2_ctx* c, int j) {
  if (!c->prm.record_masks) return;
  if ((int)c->recs.size() <= j) c->recs.resize(j + 1);
  Rec& r = c->recs[j];
  r.nnzb = c->X.nnzb;
  c->ensure(r.brow, (size_t)std::max<int64_t>(r.nnzb, 1) * 4);
  c->ensure(r.bcol, (size_t)std::max<int64_t>(r.nnzb, 1) * 4);
  c->ensure(r.rowptr, (size_t)(c->nb + 1) * 4);
  c->ck(launch_copy_index(c->X, r.brow.as<int32_t>(), r.bcol.as<int32_t>(), c->st), "record index");
  c->ck(launch_rowptr_from_brow(r.brow.as<int32_t>(), r.nnzb, c->nb, r.rowptr.as<int32_t>(), c->st), "rowptr");
  r.has_val = (j % c->prm.ckpt_every) == 0;
  if (r.has_val) {
    c->ensure(r.val, (size_t)std::max<int64_t>(r.nnzb, 1) * TE * 8);
    c->ck(launch_gather_tiles(c->X, c->pool[c->cur].as<double>(), r.val.as<double>(), c->st), "checkpoint");
  }
}

TileSet rec_tiles(sp2_ctx* c, int j) {
  Rec& r = c->recs[j];
  TileSet t;
  t.nnzb = r.nnzb;
  t.brow = r.brow.as<int32_t>();
  t.bcol = r.bcol.as<int32_t>();
  t.slot = c->ident.as<int32_t>();
  t.rowptr = r.rowptr.as<int32_t>();
  return t;
}

bool use_tc(const sp2_ctx* c, int i) {
  const sp2_params& p = c->prm;
  if (p.precision != SP2_PREC_SPLIT16) return false;
  if (i < p.mixed_from) return false;
  if (p.mixed_until > 0 && i > p.mixed_until) return false;
  if (c->tail_from > 0 && i >= c->tail_from) return false;
  // idempotency stop: the last four squares up to the iteration limit are FP64
  // too (each pair of FP64 steps squares the tensor path's rounding left on
  // both spectral sides)
  if (p.stop == SP2_STOP_IDEMPOTENCY && p.fp64_tail > 0.0 && i >= c->sch.n_max - 2) return false;
  return true;
}

// FP16 slices (scale: power of two applied before slicing) of the tiles of `x`
// (values by slot in `pool`) into `slices`, plus the super-row bitmap of `fp`.
// Panel records of the tiles of `x` (values at pool slot x.slot[t] of tile
// index t) on its both-triangle pattern `fp`: super-row bitmaps, record
// offsets, record index words, then the FP16 slices and header of every
// record.  Reads the number of records back (one host round trip).  With
// dsq: also the squared row norms of x into dsq (n doubles; FP64, unscaled).
TcOp prepare_operand(sp2_ctx* c, const TileSet& x, const double* pool, const FullPattern& fp, OpBufs& ob,
                     double scale, double* dsq = nullptr) {
  const int k = c->prm.slices;
  const int nsr = (c->nb + 3) / 4;
  const int64_t nw = (int64_t)nsr * c->words;
  c->ensure(ob.sbits, (size_t)nw * 4);
  c->ck(launch_super_bits(fp, c->nb, nsr, ob.sbits.as<uint32_t>(), c->st), "super bits");
  c->ensure(ob.cnt, (size_t)nw * 4);
  c->ensure(ob.spos, (size_t)(nw + 1) * 4);
  c->ensure(c->scantmp, scan_tmp_bytes(nw) + 4096);
  c->ck(launch_popc_words(ob.sbits.as<uint32_t>(), nw, ob.cnt.as<int32_t>(), c->st), "popc");
  c->ck(launch_scan_i32(ob.cnt.as<int32_t>(), ob.spos.as<int32_t>(), nw, ob.spos.as<int32_t>() + nw, c->scantmp.p,
                        c->st),
        "scan");
  const int64_t nrec = read_count(c, ob.spos.as<int32_t>() + nw);
  const size_t nr = (size_t)std::max<int64_t>(nrec, 1);
  c->ensure(ob.index, nr * 16);
  c->ensure(ob.head, nr);
  c->ensure(ob.data, nr * panel_record_bytes(k));
  if (nrec > 0) {
    c->ck(cudaMemsetAsync(ob.index.p, 0xFF, (size_t)nrec * 16, c->st), "memset");
    c->ck(launch_panel_fill(fp, c->nb, ob.sbits.as<uint32_t>(), ob.spos.as<int32_t>(), ob.index.as<uint32_t>(),
                            c->st),
          "record index");
    if (dsq) c->ensure(c->rsq, nr * 128 * 8);
    c->ck(launch_panel_slices(ob.index.as<uint32_t>(), nrec, x.slot, pool, ob.data.p, ob.head.as<uint8_t>(), k,
                              c->errflag.as<int32_t>(), dsq ? c->rsq.as<double>() : nullptr, scale,
                              c->selftest_pending == 2, c->st),
          "record slices");
    if (c->selftest_pending == 2) c->selftest_pending = 0;
    if (dsq)
      c->ck(launch_row_sq_sum(ob.spos.as<int32_t>(), nsr, c->words, c->rsq.as<double>(), c->n, dsq, c->st),
            "row norms");
  } else if (dsq) {
    c->ck(cudaMemsetAsync(dsq, 0, (size_t)c->n * 8, c->st), "memset");
  }
  TcOp op;
  op.sbits = ob.sbits.as<uint32_t>();
  op.spos = ob.spos.as<int32_t>();
  op.head = ob.head.as<uint8_t>();
  op.data = ob.data.p;
  return op;
}

// Smallest power of two >= max |x| over the tiles of `x` (1 for an all-zero set).
double pow2_scale(sp2_ctx* c, const TileSet& x, const double* pool) {
  c->ensure(c->amax, 16);
  c->ck(launch_absmax(x, pool, c->amax.as<unsigned long long>(), c->st), "absmax");
  c->ck(cudaMemcpyAsync(c->h_d2, c->amax.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
  c->sync();
  const double m = c->h_d2[0];
  if (!(m > 0.0) || !std::isfinite(m)) return 1.0;
  int e = 0;
  std::frexp(m, &e);            // m = f * 2^e, f in [0.5, 1)
  return std::ldexp(1.0, e);    // 2^e > m
}

// Run the tcgen05 kernel on the output tiles given by the upper bitmap `obits`
// (row offsets `orowptr`); L carries operands, coefficients and pools.
void run_tc(sp2_ctx* c, TcLaunch& L, const uint32_t* obits, const int32_t* orowptr) {
  const int k = c->prm.slices;
  const int nsr = (c->nb + 3) / 4;
  const int64_t npair = super_order_size(nsr);
  c->ensure(c->sflag, (size_t)npair * 4);
  c->ensure(c->spos, (size_t)npair * 4);
  c->ensure(c->scantmp, scan_tmp_bytes(npair) + 4096);
  c->ck(launch_super_flags(obits, c->nb, c->words, nsr, c->sflag.as<int32_t>(), c->st, L.general), "super flags");
  c->ensure(c->scount, 16);
  c->ck(launch_scan_i32(c->sflag.as<int32_t>(), c->spos.as<int32_t>(), npair, c->scount.as<int32_t>(),
                        c->scantmp.p, c->st),
        "scan");
  // no host round trip: a persistent kernel with one CTA per SM reads the
  // number of active super-tiles and takes them from a work counter
  const int64_t ubound = L.general ? (int64_t)nsr * nsr : (int64_t)nsr * (nsr + 1) / 2;
  c->ensure(c->slist, (size_t)std::max<int64_t>(ubound, 1) * 4);
  c->ck(cudaMemsetAsync(c->scount.as<int32_t>() + 1, 0, 4, c->st), "memset");
  int sms = 0;
  c->ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0), "attribute");
  const int64_t nsuper = std::min<int64_t>(std::max(sms, 1), std::max<int64_t>(ubound, 1));
  c->ck(launch_super_fill(c->sflag.as<int32_t>(), c->spos.as<int32_t>(), npair, nsr, c->slist.as<int32_t>(), c->st),
        "super fill");
  L.obits = obits;
  L.orowptr = orowptr;
  L.list = c->slist.as<int32_t>();
  L.count = c->scount.as<int32_t>();
  L.work = c->scount.as<int32_t>() + 1;
  L.nsuper = nsuper;
  L.n = c->n;
  L.nb = c->nb;
  L.nsr = nsr;
  L.k = k;
  L.words = c->words;
  c->ensure(c->tcscratch, (size_t)nsuper * tc_tile_slots() * 128 * 128 * 8);
  L.scratch = c->tcscratch.p;
  L.seg_min = c->prm.acc_flush_min;
  L.wait_ns = (unsigned long long)c->prm.wait_limit_ms * 1000000ull;
  L.split_supply = c->prm.split_supply != 0;
  L.selftest = c->selftest_pending == 1;
  if (c->selftest_pending == 1) c->selftest_pending = 0;
  L.err = c->errflag.as<int32_t>();
  if (c->prm.slices == 5 && !L.two_pass) {
    // five slices: the finest group (s + t = 4) first, its exact sum left in
    // the output tiles; then groups 0-3, added to it in the full epilogue
    // (TMEM holds four group accumulators at a time).  Every K loop is
    // accumulated in segments of 8 K tiles: 256 products of up to 2^22 per
    // element and group keep the FP32 group sums exact for dense operands,
    // which the finer grid needs to pay off.
    L.seg_min = 1;
    L.seg_ksteps = 8;
    c->ck(cudaEventRecord(c->evs0, c->st), "event");
    TcLaunch Lf = L;
    Lf.glo = 4; Lf.ghi = 4; Lf.emode = 1;
    c->ck(launch_square_tc(Lf, c->st), "square tc (finest group)");
    c->ck(cudaMemsetAsync(c->scount.as<int32_t>() + 1, 0, 4, c->st), "memset");
    TcLaunch Lm = L;
    Lm.glo = 0; Lm.ghi = 3; Lm.emode = 2;
    c->ck(launch_square_tc(Lm, c->st), "square tc");
    c->ck(cudaEventRecord(c->evs1, c->st), "event");
    return;
  }
  c->ck(cudaEventRecord(c->evs0, c->st), "event");
  c->ck(launch_square_tc(L, c->st), "square tc");
  c->ck(cudaEventRecord(c->evs1, c->st), "event");
}

// Forward: S = X~^2 on the product pattern (o_bits, upper only) with the fused epilogue.
void square_tc(sp2_ctx* c, double c0, double c1, double c2, double* outpool, bool general) {
  TcLaunch L{};
  // the diagonal of S = X~^2 from the FP64 squared row norms of X~, summed
  // while the records of A are sliced
  c->ensure(c->dsq, (size_t)c->n * 8);
  L.P = prepare_operand(c, c->X, c->pool[c->cur].as<double>(), c->fp, c->opx, 1.0, c->dsq.as<double>());
  // general storage: B is read by columns, from its own records
  L.Q = general ? prepare_operand(c, c->X, c->pool[c->cur].as<double>(), c->fpB, c->opy, 1.0) : L.P;
  L.general = general;
  L.dsq = c->dsq.as<double>();
  L.two_pass = false;
  L.scale = 1.0;
  L.Z = &c->fp;
  L.zslot = c->X.slot;
  L.zpool = c->pool[c->cur].as<double>();
  L.opool = outpool;
  L.part = partials(c);
  L.c0 = c0; L.c1 = c1; L.c2 = c2;
  run_tc(c, L, c->o_bits.as<uint32_t>(), c->o_rowptr.as<int32_t>());
}

int fill_stats_sched(sp2_ctx* c) {
  sp2_stats& s = c->stats;
  s.n_min = c->sch.n_min;
  s.n_max = c->sch.n_max;
  s.lmin = c->sch.lmin;
  s.lmax = c->sch.lmax;
  for (int i = 0; i < SP2_MAX_ITER; ++i) {
    s.p[i] = i < (int)c->sch.p.size() ? c->sch.p[i] : -1;
    s.alpha[i] = i < (int)c->sch.alpha.size() ? c->sch.alpha[i] : NAN;
    s.tau[i] = i < (int)c->sch.tau.size() ? c->sch.tau[i] : NAN;
  }
  return 0;
}

int guard(sp2_ctx* c, int code) {
  if (c) c->stats.status = code;
  return code;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int sp2_default_params(sp2_params* p) {
  if (!p) return SP2_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->mode = SP2_MODE_SP2ACC;
  p->stop = SP2_STOP_PARAMETERLESS;
  p->idem_tol = 1e-12;
  p->trunc = SP2_TRUNC_FROBENIUS;
  p->frobinf_part = 4096;
  p->gamma = 0.0;
  p->delta_acc = 0.1;
  p->n_max_cap = 100;
  p->precision = SP2_PREC_FP64;
  p->slices = 4;
  p->mixed_from = 1;
  p->mixed_until = 0;
  p->ckpt_every = 8;
  p->record_masks = 0;
  p->fp64_tail = 1e-4;
  p->acc_flush_min = 512;
  p->wait_limit_ms = 2000;
  p->selftest = 0;
  p->storage = SP2_STORAGE_SYMMETRIC;
  p->split_supply = 0;
  return SP2_OK;
}

int sp2_release_memory(void) {
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    for (HostBlock* b : g_host_free) cudaFreeHost(b);
    g_host_free.clear();
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  int rc = SP2_OK;
  for (int d = 0; d < kMaxDevices; ++d) {
    if (!g_pool[d]) continue;
    if (cudaSetDevice(d) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) {
      cudaGetLastError();
      rc = SP2_ERR_CUDA;
    }
  }
  if (cudaSetDevice(prev) != cudaSuccess) {
    cudaGetLastError();
    rc = SP2_ERR_CUDA;
  }
  return rc;
}

const char* sp2_strerror(int code) {
  switch (code) {
    case SP2_OK: return "ok";
    case SP2_ERR_INVALID_ARG: return "invalid argument";
    case SP2_ERR_BOUNDS: return "invalid homo/lumo bounds";
    case SP2_ERR_PATTERN: return "invalid tile pattern";
    case SP2_ERR_NONFINITE: return "non-finite value in input";
    case SP2_ERR_OOM: return "device allocation failed";
    case SP2_ERR_CUDA: return "CUDA error";
    case SP2_ERR_NOT_CONVERGED: return "not converged within n_max iterations";
    case SP2_ERR_TIMEOUT: return "bounded device wait timed out";
    case SP2_ERR_STATE: return "call out of order";
    case SP2_ERR_CAPACITY: return "buffer too small";
    case SP2_ERR_TOO_LARGE: return "input exceeds the fixed scratch of the allocation-free entry point";
    case SP2_ERR_RANGE: return "an iterate left the range of the method (bounds do not bracket the gap, or divergence)";
    default: return "unknown error";
  }
}

}  // extern "C"

namespace {

// Argument checks shared by sp2_create and sp2_create_dense; fills prm.
int check_create_args(int64_t n, double homo_ub, double lumo_lb, double tau, const sp2_params* params,
                      const sp2_allocator* alloc, sp2_params& prm) {
  if (n <= 0) return SP2_ERR_INVALID_ARG;
  sp2_default_params(&prm);
  if (params) prm = *params;
  if (prm.mode != SP2_MODE_SP2 && prm.mode != SP2_MODE_SP2ACC && prm.mode != SP2_MODE_TRACE)
    return SP2_ERR_INVALID_ARG;
  if (!std::isfinite(tau) || tau < 0.0) return SP2_ERR_INVALID_ARG;
  if (prm.mode == SP2_MODE_TRACE) {
    if (prm.gamma != 0.0) return SP2_ERR_INVALID_ARG;   // Eq. (7) needs a gap bound
  } else {
    if (!std::isfinite(homo_ub) || !std::isfinite(lumo_lb)) return SP2_ERR_INVALID_ARG;
    if (!(homo_ub < lumo_lb)) return SP2_ERR_BOUNDS;
  }
  if (alloc && (!alloc->alloc || !alloc->free)) return SP2_ERR_INVALID_ARG;
  if (prm.stop != SP2_STOP_PARAMETERLESS && prm.stop != SP2_STOP_IDEMPOTENCY) return SP2_ERR_INVALID_ARG;
  if (!(prm.fp64_tail >= 0.0) || !std::isfinite(prm.fp64_tail)) return SP2_ERR_INVALID_ARG;
  if (prm.acc_flush_min < 0) return SP2_ERR_INVALID_ARG;
  if (prm.trunc != SP2_TRUNC_FROBENIUS && prm.trunc != SP2_TRUNC_FROBINF && prm.trunc != SP2_TRUNC_MIXED)
    return SP2_ERR_INVALID_ARG;
  if (prm.trunc != SP2_TRUNC_FROBENIUS && (prm.frobinf_part < TB || prm.frobinf_part % TB)) return SP2_ERR_INVALID_ARG;
  if (prm.n_max_cap < 1 || prm.n_max_cap > SP2_MAX_ITER - 2) return SP2_ERR_INVALID_ARG;
  if (prm.precision != SP2_PREC_FP64 && prm.precision != SP2_PREC_SPLIT16) return SP2_ERR_INVALID_ARG;
  if (prm.precision == SP2_PREC_SPLIT16 && (prm.slices < 2 || prm.slices > 5)) return SP2_ERR_INVALID_ARG;
  if (prm.precision == SP2_PREC_SPLIT16 && prm.slices == 5 && prm.record_masks) return SP2_ERR_INVALID_ARG;
  if (prm.ckpt_every < 1) return SP2_ERR_INVALID_ARG;
  if (prm.wait_limit_ms < 1 || prm.selftest < 0 || prm.selftest > 2) return SP2_ERR_INVALID_ARG;
  if (prm.storage != SP2_STORAGE_SYMMETRIC && prm.storage != SP2_STORAGE_GENERAL) return SP2_ERR_INVALID_ARG;
  if (prm.split_supply != 0 && prm.split_supply != 1) return SP2_ERR_INVALID_ARG;
  if (prm.storage == SP2_STORAGE_GENERAL && prm.record_masks) return SP2_ERR_INVALID_ARG;
  const int64_t nb64 = (n + TB - 1) / TB;
  if (nb64 > 65535) return SP2_ERR_INVALID_ARG;
  if (prm.trunc == SP2_TRUNC_MIXED) {
    const int64_t pt = prm.frobinf_part / TB;
    if ((nb64 + pt - 1) / pt > MIXED_MAX_BLOCKS) return SP2_ERR_INVALID_ARG;
  }
  return SP2_OK;
}

sp2_ctx* new_ctx(const sp2_params& prm, const sp2_allocator* alloc, void* cuda_stream, int64_t n, int64_t nocc,
                 double homo_ub, double lumo_lb, double tau) {
  sp2_ctx* c = new (std::nothrow) sp2_ctx();
  if (!c) return nullptr;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  c->al.st = c->st;
  if (alloc) {
    c->al.a = *alloc;
    c->al.custom = true;
  } else {
    c->al.pool = device_pool();
  }
  c->prm = prm;
  c->selftest_pending = prm.selftest;
  c->n = n;
  c->nb = (int)((n + TB - 1) / TB);
  c->words = (c->nb + 31) / 32;
  c->nocc = nocc;
  c->homo_ub = homo_ub;
  c->lumo_lb = lumo_lb;
  c->tau = tau;
  return c;
}

void init_ctx_resources(sp2_ctx* c) {
  c->ck(cudaEventCreate(&c->ev0), "event");
  c->ck(cudaEventCreate(&c->ev1), "event");
  c->ck(cudaEventCreate(&c->evs0), "event");
  c->ck(cudaEventCreate(&c->evs1), "event");
  c->hb = take_host_block();
  if (!c->hb) {
    c->last_error = "page-locked host allocation failed";
    throw Fail{SP2_ERR_OOM};
  }
  c->h_sc = &c->hb->sc;
  c->h_cnt = c->hb->cnt;
  c->h_d2 = c->hb->d2;
}

// F's nnzb tiles are in f_brow / f_bcol / f_pool: validate them, then Step 1
// of Section 4 (Gershgorin bounds, schedule).
void finish_create(sp2_ctx* c, int64_t nnzb) {
  c->ensure(c->dcnt, 16);
  c->ck(launch_check_pattern(c->f_brow.as<int32_t>(), c->f_bcol.as<int32_t>(), nnzb, c->nb, c->f_pool.as<double>(),
                             c->n, c->dcnt.as<int32_t>(), c->st),
        "check");
  c->ck(cudaMemcpyAsync(c->h_cnt, c->dcnt.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
  c->sync();
  if (c->h_cnt[0] & 1) throw Fail{SP2_ERR_PATTERN};
  if (c->h_cnt[1] != c->nb) throw Fail{SP2_ERR_PATTERN};
  if (c->h_cnt[0] & 2) throw Fail{SP2_ERR_NONFINITE};
  // slots of F are the identity
  c->ensure(c->f_slot, nnzb * 4);
  c->ensure(c->f_rowptr, (c->nb + 1) * 4);
  c->ck(launch_iota(c->f_slot.as<int32_t>(), nnzb, c->st), "slots");
  set_tiles(c->F, c->f_brow, c->f_bcol, c->f_slot, c->f_rowptr, nnzb);
  c->ck(launch_rowptr_from_brow(c->F.brow, nnzb, c->nb, c->F.rowptr, c->st), "rowptr");
  // Gershgorin (Section 4, Step 1)
  build_full(c, c->F, c->fp, c->fp_bits, c->fp_rowptr, c->fp_col, c->fp_ref);
  c->ensure(c->rowlo, c->n * 8);
  c->ensure(c->rowhi, c->n * 8);
  c->ensure(c->d2, 16);
  c->ck(launch_gershgorin(c->fp, c->f_pool.as<double>(), c->nb, c->n, c->rowlo.as<double>(), c->rowhi.as<double>(),
                          c->st),
        "gershgorin");
  c->ck(launch_minmax(c->rowlo.as<double>(), c->rowhi.as<double>(), c->n, c->d2.as<double>(), c->st), "minmax");
  c->ck(cudaMemcpyAsync(c->h_d2, c->d2.p, 16, cudaMemcpyDeviceToHost, c->st), "d2h");
  c->sync();
  const double lmin = c->h_d2[0], lmax = c->h_d2[1];
  const sp2_params& prm = c->prm;
  if (prm.mode == SP2_MODE_TRACE) {
    if (!(lmax > lmin)) throw Fail{SP2_ERR_BOUNDS};
    c->sch = make_schedule_trace(lmin, lmax, c->tau, prm.n_max_cap);
  } else {
    if (!(lmin <= c->homo_ub) || !(c->lumo_lb <= lmax) || !(lmax > lmin)) throw Fail{SP2_ERR_BOUNDS};
    c->sch = make_schedule(lmin, lmax, c->homo_ub, c->lumo_lb, c->tau, prm.gamma, prm.mode == SP2_MODE_SP2ACC,
                           prm.delta_acc, prm.n_max_cap);
  }
  fill_stats_sched(c);
  c->stats.status = SP2_OK;
  c->stats.homo_est = c->stats.lumo_est = NAN;
}

int create_fail(sp2_ctx* c, const Fail& f) {
  if (f.code == SP2_ERR_CUDA || f.code == SP2_ERR_OOM) fprintf(stderr, "sp2_create: %s\n", c->last_error.c_str());
  sp2_destroy(c);
  return f.code;
}

}  // namespace

extern "C" {

int sp2_create(const sp2_bsr* F, int64_t nocc, double homo_ub, double lumo_lb, double tau,
               const sp2_params* params, const sp2_allocator* alloc, void* cuda_stream, sp2_ctx** out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!F || F->b != TB || F->n <= 0 || F->nnzb <= 0 || !F->brow || !F->bcol || !F->val) return SP2_ERR_INVALID_ARG;
  sp2_params prm;
  const int rc = check_create_args(F->n, homo_ub, lumo_lb, tau, params, alloc, prm);
  if (rc != SP2_OK) return rc;
  sp2_ctx* c = new_ctx(prm, alloc, cuda_stream, F->n, nocc, homo_ub, lumo_lb, tau);
  if (!c) return SP2_ERR_OOM;
  try {
    init_ctx_resources(c);
    const int64_t nnzb = F->nnzb;
    const cudaMemcpyKind kind = F->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->ensure(c->f_brow, nnzb * 4);
    c->ensure(c->f_bcol, nnzb * 4);
    c->ensure(c->f_pool, (size_t)nnzb * TE * 8);
    c->ck(cudaMemcpyAsync(c->f_brow.p, F->brow, nnzb * 4, kind, c->st), "copy F");
    c->ck(cudaMemcpyAsync(c->f_bcol.p, F->bcol, nnzb * 4, kind, c->st), "copy F");
    c->ck(cudaMemcpyAsync(c->f_pool.p, F->val, (size_t)nnzb * TE * 8, kind, c->st), "copy F");
    finish_create(c, nnzb);
  } catch (const Fail& f) {
    return create_fail(c, f);
  }
  *out = c;
  return SP2_OK;
}

int sp2_create_dense(const double* F, int64_t n, int64_t ld, int32_t on_device, int64_t nocc, double homo_ub,
                     double lumo_lb, double tau, const sp2_params* params, const sp2_allocator* alloc,
                     void* cuda_stream, sp2_ctx** out) {
  if (!out) return SP2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!F || n <= 0 || ld < n) return SP2_ERR_INVALID_ARG;
  sp2_params prm;
  const int rc = check_create_args(n, homo_ub, lumo_lb, tau, params, alloc, prm);
  if (rc != SP2_OK) return rc;
  const int64_t nb64 = (n + TB - 1) / TB;
  if (nb64 * nb64 >= (int64_t)1 << 31) return SP2_ERR_INVALID_ARG;   // tile flags are indexed by int32
  sp2_ctx* c = new_ctx(prm, alloc, cuda_stream, n, nocc, homo_ub, lumo_lb, tau);
  if (!c) return SP2_ERR_OOM;
  void* tmp = nullptr;
  try {
    init_ctx_resources(c);
    const double* dF = F;
    int64_t dld = ld;
    if (!on_device) {
      // device copy of the host matrix (leading dimension n)
      tmp = c->al.get((size_t)n * n * 8);
      if (!tmp) {
        c->last_error = "device allocation of the dense F copy failed";
        throw Fail{SP2_ERR_OOM};
      }
      c->ck(cudaMemcpy2DAsync(tmp, (size_t)n * 8, F, (size_t)ld * 8, (size_t)n * 8, (size_t)n,
                              cudaMemcpyHostToDevice, c->st),
            "copy F");
      dF = static_cast<const double*>(tmp);
      dld = n;
    }
    const int nb = c->nb;
    const int64_t nflag = (int64_t)nb * nb;
    c->ensure(c->scanbuf, (size_t)nflag * 4);   // tile flags
    c->ensure(c->keep, (size_t)nflag * 4);      // their exclusive scan
    c->ensure(c->dcnt, 16);
    c->ensure(c->scantmp, scan_tmp_bytes(nflag) + 4096);
    c->ck(launch_dense_tile_flags(dF, n, dld, nb, c->scanbuf.as<int32_t>(), c->st), "tile flags");
    c->ck(launch_scan_i32(c->scanbuf.as<int32_t>(), c->keep.as<int32_t>(), nflag, c->dcnt.as<int32_t>(),
                          c->scantmp.p, c->st),
          "scan");
    const int64_t nnzb = read_count(c, c->dcnt.as<int32_t>());
    c->ensure(c->f_brow, nnzb * 4);
    c->ensure(c->f_bcol, nnzb * 4);
    c->ensure(c->f_pool, (size_t)nnzb * TE * 8);
    c->ck(launch_dense_tile_fill(dF, n, dld, nb, c->scanbuf.as<int32_t>(), c->keep.as<int32_t>(),
                                 c->f_brow.as<int32_t>(), c->f_bcol.as<int32_t>(), c->f_pool.as<double>(), c->st),
          "tile fill");
    if (tmp) {
      c->al.put(tmp);
      tmp = nullptr;
    }
    finish_create(c, nnzb);
  } catch (const Fail& f) {
    if (tmp) c->al.put(tmp);
    return create_fail(c, f);
  }
  *out = c;
  return SP2_OK;
}

int sp2_run(sp2_ctx* c, sp2_stats* stats_out) {
  if (!c) return SP2_ERR_INVALID_ARG;
  int status = SP2_OK;
  try {
    sp2_stats& S = c->stats;
    const Schedule& sch = c->sch;
    if (c->prm.mode == SP2_MODE_TRACE) std::fill(c->sch.p.begin() + 1, c->sch.p.end(), -1);   // chosen below
    fill_stats_sched(c);
    S.converged = 0;
    S.squares = 0;
    S.tile_triplets = 0;
    S.square_ms = 0.0;
    S.tc_hw_flops = 0.0;
    S.have_estimates = 0;
    S.homo_est = S.lumo_est = NAN;
    for (int i = 0; i < SP2_MAX_ITER; ++i) {
      S.e[i] = S.t[i] = NAN;
      S.nnzb_hist[i] = -1;
      S.prec_hist[i] = -1;
    }
    const long long launches0 = g_launches;
    c->ensure(c->errflag, 32);
    c->ck(cudaMemsetAsync(c->errflag.p, 0, 32, c->st), "memset");
    c->ck(cudaEventRecord(c->ev0, c->st), "event");
    // Algorithm 1: X_0 on F's pattern, then X~_0 = trunc(X_0, tau_0)
    const int64_t nF = c->F.nnzb;
    c->ensure(c->pool[0], (size_t)nF * TE * 8);
    ensure_partials(c, nF);
    c->ck(launch_x0(c->F, c->f_pool.as<double>(), c->pool[0].as<double>(), c->n, sch.lmax, sch.lmax - sch.lmin,
                    c->p_n2.as<double>(), c->st),
          "x0");
    c->cur = 0;
    const bool trace_mode = c->prm.mode == SP2_MODE_TRACE;
    {
      TileSet t0 = truncate_launch(c, c->F, c->p_n2.as<double>(), sch.tau[0], 0);
      if (trace_mode) {
        // trace(X~_0) for the first choice (X_0's tiles in F's order, values in pool[0])
        c->ensure(c->trbuf, 16);
        c->ck(launch_trace_kept(c->F, c->keep.as<int32_t>(), c->pool[0].as<double>(), c->nb, c->n,
                                c->trbuf.as<double>(), c->st),
              "trace");
        c->ck(cudaMemcpyAsync(c->h_d2 + 1, c->trbuf.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
      }
      adopt_X(c, t0, read_count(c, c->dcnt.as<int32_t>()), 0);
    }
    double tr_cur = trace_mode ? c->h_d2[1] : 0.0;   // trace(X~_{i-1}) in trace mode
    const bool general = c->prm.storage == SP2_STORAGE_GENERAL;
    if (general) expand_to_general(c);
    S.nnzb_hist[0] = c->X.nnzb;
    c->tail_from = 0;
    free_recs(c);
    record(c, 0);
    std::vector<double> ev, tv;
    int n_out = -1;
    bool converged = false;
    for (int i = 1; i <= sch.n_max + 1; ++i) {
      const bool tc = use_tc(c, i);
      // symbolic: both-triangle pattern of X~_{i-1}, product pattern (upper + diagonal);
      // the tensor path addresses tiles by compact index (slices), the FP64 path by slot
      if (general) {
        build_general(c, tc);
      } else {
        TileSet Xc = c->X;
        if (tc) {
          ensure_ident(c, c->X.nnzb);
          Xc.slot = c->ident.as<int32_t>();
        }
        build_full(c, Xc, c->fp, c->fp_bits, c->fp_rowptr, c->fp_col, c->fp_ref);
      }
      c->ensure(c->o_bits, (size_t)c->nb * c->words * 4);
      c->ensure(c->o_rowptr, (size_t)(c->nb + 1) * 4);
      c->ensure(c->counts, (size_t)(c->nb + 1) * 4);
      c->ensure(c->scantmp, scan_tmp_bytes(c->nb + 1) + 4096);
      c->ck(launch_product_bits(c->fp, c->fp, c->nb, c->o_bits.as<uint32_t>(), c->st, !general), "product bits");
      c->ck(launch_row_popc(c->o_bits.as<uint32_t>(), c->nb, c->words, c->counts.as<int32_t>(), c->st), "popc");
      c->ck(launch_scan_i32(c->counts.as<int32_t>(), c->o_rowptr.as<int32_t>(), c->nb,
                            c->o_rowptr.as<int32_t>() + c->nb, c->scantmp.p, c->st),
            "scan");
      const int64_t nout = read_count(c, c->o_rowptr.as<int32_t>() + c->nb);
      c->ensure(c->o_brow, nout * 4);
      c->ensure(c->o_bcol, nout * 4);
      c->ensure(c->o_slot, nout * 4);
      set_tiles(c->out, c->o_brow, c->o_bcol, c->o_slot, c->o_rowptr, nout);
      c->ck(launch_fill_upper_from_bits(c->o_bits.as<uint32_t>(), c->nb, c->words, c->out.rowptr, c->out.brow,
                                        c->out.bcol, c->out.slot, c->st),
            "fill upper");
      const int nxt = 1 - c->cur;
      c->ensure(c->pool[nxt], (size_t)nout * TE * 8);
      ensure_partials(c, nout);
      int p = 1;
      double a = 1.0;
      if (i <= sch.n_max) {
        if (trace_mode) {
          // Section 1: x^2 lowers the trace, 2x - x^2 raises it (ties: 2x - x^2)
          c->sch.p[i] = tr_cur > (double)c->nocc ? 1 : 0;
          S.p[i] = c->sch.p[i];
        }
        p = sch.p[i];
        a = sch.alpha[i];
      }
      double c0, c1, c2;
      coeffs(p, a, c0, c1, c2);
      SquareArgs sa;
      sa.A = &c->fp; sa.apool = c->pool[c->cur].as<double>();
      sa.B = general ? &c->fpB : &c->fp; sa.bpool = sa.apool;
      sa.sym_sum = false;
      sa.general = general;
      sa.Z = &c->fp; sa.zpool = sa.apool;
      sa.out = &c->out; sa.outpool = c->pool[nxt].as<double>();
      sa.c0 = c0; sa.c1 = c1; sa.c2 = c2;
      sa.n = c->n; sa.nb = c->nb;
      sa.part = partials(c);
      if (tc) {
        square_tc(c, c0, c1, c2, sa.outpool, general);
      } else {
        c->ck(cudaEventRecord(c->evs0, c->st), "event");
        c->ck(launch_square_f64(sa, c->st), "square f64");
        c->ck(cudaEventRecord(c->evs1, c->st), "event");
      }
      c->ensure(c->dsc, sizeof(StepScalars));
      c->ensure(c->redwork, reduce_work_bytes());
      c->ck(launch_reduce_step(sa.part, nout, c->dsc.as<StepScalars>(), c->redwork.p, c->st), "reduce");
      // X~_i = trunc(X_i, tau_i) before the stop test on e_{i-1} is known (X_i's tiles
      // live in pool[nxt] at slot = output index); X~_{i-1} keeps its own index set
      const bool more = i <= sch.n_max;
      TileSet next;
      if (more)
        next = general ? truncate_launch_general(c, c->out, c->p_n2.as<double>(), sch.tau[i], 1 - c->xset)
                       : truncate_launch(c, c->out, c->p_n2.as<double>(), sch.tau[i], 1 - c->xset);
      if (more && trace_mode) {
        // trace(X~_i) for the next choice: the kept diagonal tiles of the output
        c->ck(launch_trace_kept(c->out, c->keep.as<int32_t>(), c->pool[nxt].as<double>(), c->nb, c->n,
                                c->trbuf.as<double>(), c->st),
              "trace");
        c->ck(cudaMemcpyAsync(c->h_d2 + 1, c->trbuf.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
      }
      // one host round trip per step: scalars, error flags, kept-tile count
      c->ck(cudaMemcpyAsync(c->h_sc, c->dsc.p, sizeof(StepScalars), cudaMemcpyDeviceToHost, c->st), "d2h");
      c->ck(cudaMemcpyAsync(c->h_cnt + 2, c->errflag.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
      c->ck(cudaMemcpyAsync(c->h_d2, c->errflag.as<char>() + 8, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
      if (more) c->ck(cudaMemcpyAsync(c->h_cnt, c->dcnt.p, 4, cudaMemcpyDeviceToHost, c->st), "d2h");
      c->sync();
      if (c->h_cnt[2] & 1) {
        char sites[16];
        snprintf(sites, sizeof sites, "0x%x", (unsigned)c->h_cnt[3]);
        c->last_error = std::string("tensor-core square: a bounded wait timed out (sites ") + sites + ")";
        fprintf(stderr, "sp2_run: %s\n", c->last_error.c_str());
        throw Fail{SP2_ERR_TIMEOUT};
      }
      if (c->h_cnt[2] & 4) {
        c->last_error = "an element of the iterate reached |x| >= 2, outside the range of the tensor-core slices";
        fprintf(stderr, "sp2_run: %s\n", c->last_error.c_str());
        throw Fail{SP2_ERR_RANGE};
      }
      if (tc) {
        // slice-pair products issued, each two 128 x 128 x 16 MMAs
        const long long products = *reinterpret_cast<long long*>(c->h_d2);
        S.tc_hw_flops = (double)products * 2.0 * 128.0 * 128.0 * 32.0;
      }
      float ms = 0.f;
      c->ck(cudaEventElapsedTime(&ms, c->evs0, c->evs1), "elapsed");
      S.square_ms += ms;
      S.squares += 1;
      S.tile_triplets += c->h_sc->triplets;
      const int j = i - 1;
      const double ej = std::sqrt(std::max(c->h_sc->e2, 0.0));
      const double tj = c->h_sc->trX - c->h_sc->trS;
      if (!std::isfinite(ej) || !std::isfinite(tj)) {
        c->last_error = "e_j or t_j is not finite";
        fprintf(stderr, "sp2_run: %s\n", c->last_error.c_str());
        throw Fail{SP2_ERR_RANGE};
      }
      ev.push_back(ej);
      tv.push_back(tj);
      S.e[j] = ej;
      S.t[j] = tj;
      S.prec_hist[j] = tc ? SP2_PREC_SPLIT16 : SP2_PREC_FP64;
      // the final idempotency steps run in FP64 (SPLIT16 with the idempotency stop)
      if (c->prm.stop == SP2_STOP_IDEMPOTENCY && c->prm.fp64_tail > 0.0 && ej < c->prm.fp64_tail &&
          c->tail_from == 0)
        c->tail_from = i + 1;
      bool stop = false;
      if (c->prm.stop == SP2_STOP_PARAMETERLESS) {
        stop = j >= std::max(sch.n_min, 2) && sch.p[j] != sch.p[j - 1] && ev[j] > C_STOP * (ev[j - 2] * ev[j - 2]);
      } else {
        stop = ev[j] < c->prm.idem_tol;
      }
      if (stop) { n_out = j; converged = true; break; }
      if (!more) { n_out = j; break; }
      adopt_X(c, next, c->h_cnt[0], 1 - c->xset);
      if (trace_mode) tr_cur = c->h_d2[1];
      c->cur = nxt;
      S.nnzb_hist[i] = c->X.nnzb;
      record(c, i);
    }
    // D = X~_n: contiguous copy of its upper tiles for the caller's view
    TileSet Dx = c->X;
    if (general) {
      c->ensure(c->gflag, (size_t)std::max<int64_t>(c->X.nnzb, 1) * 4);
      c->ensure(c->gpos, (size_t)std::max<int64_t>(c->X.nnzb, 1) * 4);
      c->ensure(c->u_brow, (size_t)std::max<int64_t>(c->X.nnzb, 1) * 4);
      c->ensure(c->u_bcol, (size_t)std::max<int64_t>(c->X.nnzb, 1) * 4);
      c->ensure(c->u_slot, (size_t)std::max<int64_t>(c->X.nnzb, 1) * 4);
      c->ensure(c->scantmp, scan_tmp_bytes(c->X.nnzb) + 4096);
      c->ck(launch_upper_flags(c->X, c->gflag.as<int32_t>(), c->st), "upper flags");
      Dx.brow = c->u_brow.as<int32_t>();
      Dx.bcol = c->u_bcol.as<int32_t>();
      Dx.slot = c->u_slot.as<int32_t>();
      Dx.rowptr = nullptr;
      c->ck(launch_compact(c->X, c->gflag.as<int32_t>(), c->nb, Dx, c->dcnt.as<int32_t>(), c->scantmp.p,
                           c->gpos.as<int32_t>(), c->st),
            "upper tiles");
      Dx.nnzb = read_count(c, c->dcnt.as<int32_t>());
    }
    c->d_nnzb = Dx.nnzb;
    c->ensure(c->d_brow, std::max<int64_t>(c->d_nnzb, 1) * 4);
    c->ensure(c->d_bcol, std::max<int64_t>(c->d_nnzb, 1) * 4);
    c->ensure(c->d_val, (size_t)std::max<int64_t>(c->d_nnzb, 1) * TE * 8);
    c->ck(launch_copy_index(Dx, c->d_brow.as<int32_t>(), c->d_bcol.as<int32_t>(), c->st), "copy index");
    c->ck(launch_gather_tiles(Dx, c->pool[c->cur].as<double>(), c->d_val.as<double>(), c->st), "gather");
    c->ck(cudaEventRecord(c->ev1, c->st), "event");
    c->sync();
    float ms = 0.f;
    c->ck(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "elapsed");
    S.run_ms = ms;
    S.kernel_launches = g_launches - launches0;
    S.n = n_out;
    S.converged = converged ? 1 : 0;
    S.nnzb_final = c->d_nnzb;
    S.alg_flops = 2.0 * TB * TB * TB * (double)S.tile_triplets;
    double h = NAN, l = NAN;
    int have = 0;
    estimates(sch, ev, tv, c->n, h, l, have);
    S.homo_est = h;
    S.lumo_est = l;
    S.have_estimates = have;
    c->ran = true;
    c->have_D = true;
    status = converged ? SP2_OK : SP2_ERR_NOT_CONVERGED;
  } catch (const Fail& f) {
    if (f.code == SP2_ERR_CUDA || f.code == SP2_ERR_OOM) fprintf(stderr, "sp2_run: %s\n", c->last_error.c_str());
    status = f.code;
  }
  c->stats.status = status;
  if (stats_out) *stats_out = c->stats;
  return status;
}

int sp2_estimate_bounds(const sp2_ctx* c, double margin, double* homo_ub, double* lumo_lb) {
  if (!c || !homo_ub || !lumo_lb || !(margin >= 0.0) || !(margin < 0.5)) return SP2_ERR_INVALID_ARG;
  const sp2_stats& s = c->stats;
  if (!c->ran || (s.have_estimates & 3) != 3 || !(s.lumo_est > s.homo_est)) return SP2_ERR_STATE;
  const double d = margin * (s.lumo_est - s.homo_est);
  *homo_ub = std::max(s.homo_est + d, s.lmin);
  *lumo_lb = std::min(s.lumo_est - d, s.lmax);
  return SP2_OK;
}

int sp2_get_D(sp2_ctx* c, sp2_bsr* view) {
  if (!c || !view) return SP2_ERR_INVALID_ARG;
  if (!c->have_D) return SP2_ERR_STATE;
  view->n = c->n;
  view->b = TB;
  view->nnzb = c->d_nnzb;
  view->brow = c->d_brow.as<int32_t>();
  view->bcol = c->d_bcol.as<int32_t>();
  view->val = c->d_val.as<double>();
  view->on_device = 1;
  return SP2_OK;
}

int sp2_copy_D(sp2_ctx* c, int32_t* brow, int32_t* bcol, double* val, int64_t cap_nnzb, int32_t on_device,
               int64_t* nnzb_out) {
  if (!c) return SP2_ERR_INVALID_ARG;
  if (!c->have_D) return SP2_ERR_STATE;
  if (nnzb_out) *nnzb_out = c->d_nnzb;
  if (cap_nnzb < c->d_nnzb) return SP2_ERR_CAPACITY;
  if (!brow || !bcol || !val) return SP2_ERR_INVALID_ARG;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  try {
    c->ck(cudaMemcpyAsync(brow, c->d_brow.p, c->d_nnzb * 4, k, c->st), "copy D");
    c->ck(cudaMemcpyAsync(bcol, c->d_bcol.p, c->d_nnzb * 4, k, c->st), "copy D");
    c->ck(cudaMemcpyAsync(val, c->d_val.p, (size_t)c->d_nnzb * TE * 8, k, c->st), "copy D");
    c->sync();
  } catch (const Fail& f) {
    return f.code;
  }
  return SP2_OK;
}

int sp2_copy_D_dense(sp2_ctx* c, double* out, int64_t ld, int32_t on_device) {
  if (!c || !out || ld < c->n) return SP2_ERR_INVALID_ARG;
  if (!c->have_D) return SP2_ERR_STATE;
  void* tmp = nullptr;
  try {
    double* dst = out;
    int64_t dld = ld;
    if (!on_device) {
      tmp = c->al.get((size_t)c->n * c->n * 8);
      if (!tmp) {
        c->last_error = "device allocation of the dense D buffer failed";
        throw Fail{SP2_ERR_OOM};
      }
      dst = static_cast<double*>(tmp);
      dld = c->n;
    }
    c->ck(launch_tiles_to_dense(c->d_brow.as<int32_t>(), c->d_bcol.as<int32_t>(), c->d_val.as<double>(), c->d_nnzb,
                                c->n, dld, dst, c->st),
          "dense D");
    if (!on_device)
      c->ck(cudaMemcpy2DAsync(out, (size_t)ld * 8, dst, (size_t)c->n * 8, (size_t)c->n * 8, (size_t)c->n,
                              cudaMemcpyDeviceToHost, c->st),
            "copy D");
    c->sync();
    if (tmp) c->al.put(tmp);
  } catch (const Fail& f) {
    if (tmp) c->al.put(tmp);
    if (f.code == SP2_ERR_CUDA || f.code == SP2_ERR_OOM) fprintf(stderr, "sp2_copy_D_dense: %s\n", c->last_error.c_str());
    return f.code;
  }
  return SP2_OK;
}

int sp2_backward(sp2_ctx* c, const sp2_bsr* W, sp2_bsr* dF) {
  if (!c || !W || !dF) return SP2_ERR_INVALID_ARG;
  if (W->b != TB || W->n != c->n || W->nnzb < 0 || (W->nnzb > 0 && (!W->brow || !W->bcol || !W->val)))
    return SP2_ERR_INVALID_ARG;
  if (!c->have_D || !c->prm.record_masks) return SP2_ERR_STATE;
  const int n = c->stats.n;
  if (n < 0 || (int)c->recs.size() < n + 1) return SP2_ERR_STATE;
  try {
    c->ck(cudaEventRecord(c->ev0, c->st), "event");
    c->ensure(c->errflag, 32);
    c->ck(cudaMemsetAsync(c->errflag.p, 0, 32, c->st), "memset");
    const Schedule& sch = c->sch;
    const int k = c->prm.ckpt_every;
    // W -> device, validated like F (diagonal tiles not required)
    const int64_t nw = W->nnzb;
    const cudaMemcpyKind kind = W->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->ensure(c->w_brow, (size_t)std::max<int64_t>(nw, 1) * 4);
    c->ensure(c->w_bcol, (size_t)std::max<int64_t>(nw, 1) * 4);
    c->ensure(c->w_rowptr, (size_t)(c->nb + 1) * 4);
    c->ensure(c->w_pool, (size_t)std::max<int64_t>(nw, 1) * TE * 8);
    if (nw > 0) {
      c->ck(cudaMemcpyAsync(c->w_brow.p, W->brow, nw * 4, kind, c->st), "copy W");
      c->ck(cudaMemcpyAsync(c->w_bcol.p, W->bcol, nw * 4, kind, c->st), "copy W");
      c->ck(cudaMemcpyAsync(c->w_pool.p, W->val, (size_t)nw * TE * 8, kind, c->st), "copy W");
      c->ensure(c->dcnt, 16);
      c->ck(launch_check_pattern(c->w_brow.as<int32_t>(), c->w_bcol.as<int32_t>(), nw, c->nb, c->w_pool.as<double>(),
                                 c->n, c->dcnt.as<int32_t>(), c->st),
            "check W");
      c->ck(cudaMemcpyAsync(c->h_cnt, c->dcnt.p, 8, cudaMemcpyDeviceToHost, c->st), "d2h");
      c->sync();
      if (c->h_cnt[0] & 1) throw Fail{SP2_ERR_PATTERN};
      if (c->h_cnt[0] & 2) throw Fail{SP2_ERR_NONFINITE};
    }
    c->ck(launch_rowptr_from_brow(c->w_brow.as<int32_t>(), nw, c->nb, c->w_rowptr.as<int32_t>(), c->st), "rowptr");
    int64_t mx = std::max<int64_t>(nw, c->F.nnzb);
    for (int j = 0; j <= n; ++j) mx = std::max(mx, c->recs[j].nnzb);
    ensure_ident(c, mx);
    TileSet Wt;
    Wt.nnzb = nw;
    Wt.brow = c->w_brow.as<int32_t>();
    Wt.bcol = c->w_bcol.as<int32_t>();
    Wt.slot = c->ident.as<int32_t>();
    Wt.rowptr = c->w_rowptr.as<int32_t>();
    // G_n = W on the tiles of D = X~_n (dL/dD for L = trace(D W), W symmetric)
    int gcur = 0;
    {
      TileSet tn = rec_tiles(c, n);
      c->ensure(c->gpool[0], (size_t)std::max<int64_t>(tn.nnzb, 1) * TE * 8);
      c->ck(launch_place(Wt, c->w_pool.as<double>(), tn, c->gpool[0].as<double>(), 1.0, 1, c->st), "place W");
    }
    int i = n;
    while (i >= 1) {
      const int cp = ((i - 1) / k) * k;  // checkpoint holding X~_cp
      if (!c->recs[cp].has_val) throw Fail{SP2_ERR_STATE};
      // recompute X~_{cp+1} .. X~_{i-1} on their recorded tiles (no truncation needed)
      const int len = i - cp;             // seg[0] = X~_cp, ..., seg[len-1] = X~_{i-1}
      if ((int)c->seg.size() < len) c->seg.resize(len);
      std::vector<const double*> vals(len);
      vals[0] = c->recs[cp].val.as<double>();
      for (int j = cp + 1; j < i; ++j) {
        TileSet prev = rec_tiles(c, j - 1), cur = rec_tiles(c, j);
        build_full(c, prev, c->fpB, c->fpB_bits, c->fpB_rowptr, c->fpB_col, c->fpB_ref);
        Buf& dst = c->seg[j - cp];
        c->ensure(dst, (size_t)std::max<int64_t>(cur.nnzb, 1) * TE * 8);
        ensure_partials(c, std::max<int64_t>(cur.nnzb, 1));
        double c0, c1, c2;
        coeffs(sch.p[j], sch.alpha[j], c0, c1, c2);
        if (c->prm.precision == SP2_PREC_SPLIT16) {
          // X~_j on its recorded tiles: P = Q = Z = X~_{j-1}
          TcLaunch L{};
          L.P = prepare_operand(c, prev, vals[j - 1 - cp], c->fpB, c->opy, 1.0);
          L.Q = L.P;
          c->ensure(c->o_bits, (size_t)c->nb * c->words * 4);
          c->ck(launch_upper_bits(cur, c->nb, c->words, c->o_bits.as<uint32_t>(), c->st), "upper bits");
          L.two_pass = false;
          L.scale = 1.0;
          L.Z = &c->fpB;
          L.zpool = vals[j - 1 - cp];
          L.opool = dst.as<double>();
          L.part = partials(c);
          L.c0 = c0; L.c1 = c1; L.c2 = c2;
          run_tc(c, L, c->o_bits.as<uint32_t>(), cur.rowptr);
          vals[j - cp] = dst.as<double>();
          continue;
        }
        SquareArgs sa;
        sa.A = &c->fpB; sa.apool = vals[j - 1 - cp];
        sa.B = &c->fpB; sa.bpool = vals[j - 1 - cp];
        sa.sym_sum = false;
        sa.Z = &c->fpB; sa.zpool = vals[j - 1 - cp];
        sa.out = &cur; sa.outpool = dst.as<double>();
        sa.c0 = c0; sa.c1 = c1; sa.c2 = c2;
        sa.n = c->n; sa.nb = c->nb;
        sa.part = partials(c);
        c->ck(launch_square_f64(sa, c->st), "replay square");
        vals[j - cp] = dst.as<double>();
      }
      // reverse steps i .. cp+1:  G_{j-1} = mask_{j-1}( c1 G_j + c2 (G_j X~_{j-1} + X~_{j-1} G_j) )
      for (; i > cp; --i) {
        TileSet tg = rec_tiles(c, i), tp = rec_tiles(c, i - 1);
        build_full(c, tg, c->fp, c->fp_bits, c->fp_rowptr, c->fp_col, c->fp_ref);
        build_full(c, tp, c->fpB, c->fpB_bits, c->fpB_rowptr, c->fpB_col, c->fpB_ref);
        const int nxt = 1 - gcur;
        c->ensure(c->gpool[nxt], (size_t)std::max<int64_t>(tp.nnzb, 1) * TE * 8);
        ensure_partials(c, std::max<int64_t>(tp.nnzb, 1));
        double c0, c1, c2;
        coeffs(sch.p[i], sch.alpha[i], c0, c1, c2);
        if (c->prm.precision == SP2_PREC_SPLIT16) {
          // G_{i-1} on X~_{i-1}'s tiles: c1 G_i + c2 (G_i X~_{i-1} + X~_{i-1} G_i), two passes
          const double sg = pow2_scale(c, tg, c->gpool[gcur].as<double>());
          TcLaunch L{};
          L.P = prepare_operand(c, tg, c->gpool[gcur].as<double>(), c->fp, c->opx, sg);
          L.Q = prepare_operand(c, tp, vals[i - 1 - cp], c->fpB, c->opy, 1.0);
          c->ensure(c->o_bits, (size_t)c->nb * c->words * 4);
          c->ck(launch_upper_bits(tp, c->nb, c->words, c->o_bits.as<uint32_t>(), c->st), "upper bits");
          L.two_pass = true;
          L.scale = sg;
          L.Z = &c->fp;
          L.zpool = c->gpool[gcur].as<double>();
          L.opool = c->gpool[nxt].as<double>();
          L.part = partials(c);
          L.c0 = 0.0; L.c1 = c1; L.c2 = c2;
          run_tc(c, L, c->o_bits.as<uint32_t>(), tp.rowptr);
          gcur = nxt;
          continue;
        }
        SquareArgs sa;
        sa.A = &c->fp; sa.apool = c->gpool[gcur].as<double>();
        sa.B = &c->fpB; sa.bpool = vals[i - 1 - cp];
        sa.sym_sum = true;
        sa.Z = &c->fp; sa.zpool = c->gpool[gcur].as<double>();
        sa.out = &tp; sa.outpool = c->gpool[nxt].as<double>();
        sa.c0 = 0.0; sa.c1 = c1; sa.c2 = c2;
        sa.n = c->n; sa.nb = c->nb;
        sa.part = partials(c);
        c->ck(launch_square_f64(sa, c->st), "adjoint step");
        gcur = nxt;
      }
    }
    // X_0 = (lmax I - F) / w:  dL/dF = -G_0 / w on F's tiles (0 where X~_0 dropped a tile)
    TileSet t0 = rec_tiles(c, 0);
    c->ensure(c->dF, (size_t)std::max<int64_t>(c->F.nnzb, 1) * TE * 8);
    c->ck(launch_place(t0, c->gpool[gcur].as<double>(), c->F, c->dF.as<double>(), -1.0 / (sch.lmax - sch.lmin), 0,
                       c->st),
          "dF");
    c->ck(cudaEventRecord(c->ev1, c->st), "event");
    c->ck(cudaMemcpyAsync(c->h_cnt + 2, c->errflag.p, 4, cudaMemcpyDeviceToHost, c->st), "d2h");
    c->sync();
    if (c->h_cnt[2] & 1) {
      c->last_error = "tensor-core adjoint: a bounded wait timed out";
      throw Fail{SP2_ERR_TIMEOUT};
    }
    if (c->h_cnt[2] & 4) {
      c->last_error = "an element of an adjoint operand reached the edge of the tensor-core slices";
      throw Fail{SP2_ERR_RANGE};
    }
    float ms = 0.f;
    c->ck(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "elapsed");
    c->backward_ms = ms;
    c->stats.backward_ms = ms;
    dF->n = c->n;
    dF->b = TB;
    dF->nnzb = c->F.nnzb;
    dF->brow = c->F.brow;
    dF->bcol = c->F.bcol;
    dF->val = c->dF.as<double>();
    dF->on_device = 1;
  } catch (const Fail& f) {
    if (f.code == SP2_ERR_CUDA || f.code == SP2_ERR_OOM) fprintf(stderr, "sp2_backward: %s\n", c->last_error.c_str());
    return f.code;
  }
  return SP2_OK;
}

int sp2_truncate(const sp2_bsr* X, double tau, int32_t mode, int64_t frobinf_part, int32_t* keep,
                 void* cuda_stream) {
  if (!X || !keep || X->b != TB || X->n <= 0 || X->nnzb < 0 || !(tau >= 0.0) || !std::isfinite(tau))
    return SP2_ERR_INVALID_ARG;
  if (X->nnzb > 0 && (!X->brow || !X->bcol || !X->val)) return SP2_ERR_INVALID_ARG;
  if (mode != SP2_TRUNC_FROBENIUS && mode != SP2_TRUNC_FROBINF && mode != SP2_TRUNC_MIXED) return SP2_ERR_INVALID_ARG;
  if (mode != SP2_TRUNC_FROBENIUS && (frobinf_part < TB || frobinf_part % TB)) return SP2_ERR_INVALID_ARG;
  const int64_t nb64 = (X->n + TB - 1) / TB;
  if (nb64 > 65535) return SP2_ERR_INVALID_ARG;
  if (mode == SP2_TRUNC_MIXED && (nb64 + frobinf_part / TB - 1) / (frobinf_part / TB) > MIXED_MAX_BLOCKS)
    return SP2_ERR_INVALID_ARG;
  if (X->nnzb == 0) return SP2_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (int)nb64;
  const int64_t nnzb = X->nnzb;
  const int64_t part_tiles = std::max<int64_t>(1, frobinf_part / TB);
  void *dbrow = nullptr, *dbcol = nullptr, *dval = nullptr, *dn2 = nullptr, *work = nullptr, *dkeep = nullptr;
  int rc = SP2_OK;
  auto get = [&](void** p, size_t bytes) {
    if (cudaMallocAsync(p, std::max<size_t>(bytes, 256), st) != cudaSuccess) {
      cudaGetLastError();
      rc = SP2_ERR_OOM;
      return false;
    }
    return true;
  };
  const bool dev = X->on_device != 0;
  const int32_t* brow = X->brow;
  const int32_t* bcol = X->bcol;
  const double* val = X->val;
  do {
    if (!dev) {
      if (!get(&dbrow, nnzb * 4) || !get(&dbcol, nnzb * 4) || !get(&dval, (size_t)nnzb * TE * 8)) break;
      if (cudaMemcpyAsync(dbrow, X->brow, nnzb * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(dbcol, X->bcol, nnzb * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(dval, X->val, (size_t)nnzb * TE * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = SP2_ERR_CUDA;
        break;
      }
      brow = static_cast<int32_t*>(dbrow);
      bcol = static_cast<int32_t*>(dbcol);
      val = static_cast<double*>(dval);
    }
    const int nsb = (int)((nb + part_tiles - 1) / part_tiles);
    const size_t wbytes = mode == SP2_TRUNC_MIXED ? mixed_work_bytes(nnzb, nsb) : trunc_work_bytes(nnzb, nb, part_tiles);
    if (!get(&dn2, nnzb * 8) || !get(&work, wbytes)) break;
    int32_t* kout = keep;
    if (!dev) {
      if (!get(&dkeep, nnzb * 4)) break;
      kout = static_cast<int32_t*>(dkeep);
    }
    TileSet ts;
    ts.nnzb = nnzb;
    ts.brow = const_cast<int32_t*>(brow);
    ts.bcol = const_cast<int32_t*>(bcol);
    ts.slot = nullptr;
    if (launch_tile_norms(val, nnzb, static_cast<double*>(dn2), st) != cudaSuccess ||
        (mode == SP2_TRUNC_MIXED
             ? mixed_select(ts, static_cast<double*>(dn2), nb, tau, part_tiles, work, kout, st)
             : launch_truncate(ts, static_cast<double*>(dn2), nb, tau, mode, part_tiles, work, kout, st)) !=
            cudaSuccess) {
      rc = SP2_ERR_CUDA;
      break;
    }
    if (!dev && cudaMemcpyAsync(keep, dkeep, nnzb * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      rc = SP2_ERR_CUDA;
      break;
    }
  } while (false);
  for (void* p : {dbrow, dbcol, dval, dn2, work, dkeep})
    if (p) cudaFreeAsync(p, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == SP2_OK) rc = SP2_ERR_CUDA;
  return rc;
}

int sp2_get_stats(const sp2_ctx* c, sp2_stats* s) {
  if (!c || !s) return SP2_ERR_INVALID_ARG;
  *s = c->stats;
  return SP2_OK;
}

void sp2_destroy(sp2_ctx* c) {
  if (!c) return;
  free_recs(c);
  for (Buf* b : c->bufs) {
    c->al.put(b->p);
    b->p = nullptr;
  }
  cudaStreamSynchronize(c->st);
  give_host_block(c->hb);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evs0) cudaEventDestroy(c->evs0);
  if (c->evs1) cudaEventDestroy(c->evs1);
  delete c;
}

}  // extern "C"
