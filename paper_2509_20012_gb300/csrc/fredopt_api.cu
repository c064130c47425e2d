// C ABI of libfredopt (include/fredopt.h): plan upload and setup (stage
// (iii) of Table 2), the device-resident iteration of Fig. 3 around the
// simultaneous form of Fig. 2, and the final FP64 outputs.
//
// Device order of rows: with FREDOPT_ROWS_ROI the rows of voxels that belong
// to some structure come first (ascending voxel), then all other rows; the
// iteration streams only the first n_hot rows (Fig. 2 visits the voxels of
// the ROIs only).  With FREDOPT_ROWS_ALL the order is the voxel order and
// every row is streamed every pass.  The final outputs always cover every
// voxel.
#include "fredopt.h"
#include "fredopt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

using namespace fo;

namespace {

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t count) {
    release();
    const size_t c = count ? count : 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), c * sizeof(T));
    if (e == cudaSuccess) n = count;
    else p = nullptr;
    return e;
  }
  cudaError_t ensure(size_t count) { return (p && n >= count) ? cudaSuccess : alloc(count); }
};

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  int cls = 0;
};

// the two event-record nodes around one kernel of a timed iteration graph
struct GraphTimer {
  cudaGraphNode_t a = nullptr, b = nullptr;
  int cls = 0;
};

}  // namespace

struct fredopt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_join = nullptr, ev_it0 = nullptr, ev_it1 = nullptr;
  Geometry geo{};       // launch shapes of the loaded plan
  Geometry geo_full{};  // the device's full-GPU shapes
  std::string last_error;
  size_t l2_bytes = 0;

  // plan
  bool loaded = false;
  int fmt = 0;
  bool roi = false;
  int64_t V = 0, nnz = 0, n_hot = 0, nnz_hot = 0;
  int64_t n_hot_ne = 0, n_cold_ne = 0;  // rows with nonzeros among streamed / other rows
  bool perm = false;                    // device order differs from voxel order
  int32_t n = 0, n_pad = 0;
  DBuf<int64_t> rp;
  DBuf<int32_t> col;
  DBuf<uint16_t> col16;  // 16-bit copy of col for the forward stream (col then freed)
  DBuf<uint8_t> Dv, Lv;
  DBuf<float> sD, sL;
  DBuf<int64_t> voxel;  // device row -> voxel (when perm)
  DBuf<uint32_t> mask;  // [n_hot]
  DBuf<double> mdd, mll, mdl;
  DBuf<int64_t> cp;
  DBuf<int32_t> crow;
  // based 16-bit copy of crow for the transposed product (per 128-element
  // block: base row in chdr, or an overflow slot of covf for wide blocks)
  DBuf<uint16_t> crow16;
  DBuf<int32_t> chdr, covf;
  DBuf<unsigned int> cnw;
  int64_t n_wide_blocks = 0;
  DBuf<uint8_t> DTv, LTv;
  DBuf<int64_t> warp_row_hot, warp_row_all, chunk_ptr;
  DBuf<int64_t> tile_row_hot;  // claimed tiles of the streamed rows (guided sizes)
  int n_tiles_hot = 0;
  DBuf<unsigned int> fsched;   // counters of the claimed tiles
  DBuf<int32_t> tile_chunk;    // claimed tiles of the transposed product: chunk bounds [n_tiles_bwd + 1]
  int n_tiles_bwd = 0;
  DBuf<unsigned int> bsched;
  DBuf<int32_t> col_chunk, warp_chunk;
  int64_t n_chunks = 0;
  bool hint_fwd = true, hint_bwd = true;
  std::vector<int64_t> h_voxel;  // device row -> voxel (host copy, when perm)
  std::vector<int64_t> h_rp;     // row_ptr in device order (host copy, for the schedules)
  std::vector<int64_t> h_cptr;   // chunk_ptr (host copy)
  int64_t row_cost = 0, chunk_cost = 0;  // warp-partition weights in use
  std::vector<uint32_t> h_mask;  // per streamed row
  DBuf<int64_t> con_rows;        // streamed rows with a structure bit, ascending
  std::vector<int64_t> h_con_rows;
  int64_t n_con_rows = 0;
  DBuf<float2> ucoef;            // coefficients of fredopt_backward (kept apart from gam)

  // problem
  Tables tab{};
  bool have_con = false;
  bool obj_dose = false;
  double W_all = 0.0;
  int64_t n_rows_reach = 0, n_unreach = 0;

  // buffers
  DBuf<float> w, g, xbuf, gtmp;
  DBuf<float2> yw, yg, r, gam, yall;
  DBuf<double2> y64;
  DBuf<float> chunk_sum, fout_a, fout_b, vin_a, vin_b;
  DBuf<uint8_t> vol_buf;  // volume statistics scratch

  // block-iterative sweep (built for sweep_m requested blocks; 0 = not built)
  int sweep_m = 0;
  int sweep_nb = 0;                          // blocks actually formed
  std::vector<int64_t> h_sweep_bounds;       // [sweep_nb + 1] device rows
  std::vector<int64_t> sweep_wr_off;         // [sweep_nb] offset (in pairs) of each block's warp ranges
  std::vector<int> sweep_warps;              // [sweep_nb] warps of each block's forward product
  DBuf<int64_t> sweep_wr, sweep_pos, sweep_bounds_d;
  DBuf<float> xs;                            // the point being swept [n_pad]
  DBuf<float2> ys;                           // forward product of the block rows [n_hot]
  DBuf<double> part;
  // steps beta0 alpha^s of the trial loop for s < kBetaTable (in `part` at
  // off_btab), filled on the device for (btab_alpha, btab_beta0)
  double btab_alpha = -1.0, btab_beta0 = -1.0;
  DBuf<DevState> st;
  DBuf<LogEntry> log;
  DBuf<int> errw;
  size_t off_f = 0, off_bc = 0, off_g = 0, off_k2 = 0, off_fin = 0, off_cnt = 0, off_stage = 0, off_btab = 0,
         n_part = 0;

  // solve
  bool begun = false;
  fredopt_params prm{};
  double alpha = 0.99, lam = 1.0, beta0 = 0.0;
  int64_t iters_run = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_nodes = 0;
  double device_ms = 0.0;
  bool it_pending = false;
  DevState st_host{};

  // timing
  bool timing = false;
  std::vector<Timer> timers;
  size_t timers_used = 0;
  bool capturing = false;            // enqueue_iteration is being captured into `graph`
  bool graph_timed = false;          // `graph` holds an event pair around each kernel
  std::vector<GraphTimer> gtimers;   // those pairs, in kernel order
  double kms[FREDOPT_KCLASS_N] = {0};
  int64_t klaunch[FREDOPT_KCLASS_N] = {0};
  int64_t launches = 0;  // kernels enqueued (graph replays count their nodes)
};

namespace {

const char* kErrNames[] = {"ok",        "invalid argument", "shape",     "pattern",
                           "nonfinite", "not loaded",       "out of memory", "cuda error",
                           "timeout",   "unsupported"};

int fail(fredopt_t h, int code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

int cuda_fail(fredopt_t h, cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FREDOPT_ERR_OOM : FREDOPT_ERR_CUDA;
  cudaGetLastError();  // clear non-sticky errors so the handle stays usable
  return fail(h, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool dev_ptr(uint32_t flags) { return (flags & FREDOPT_DEVICE_PTR) != 0; }

// Order the handle's own stream after the legacy default stream, so device
// inputs written there by the caller are visible.
void join_in(fredopt_t h) {
  if (!h->own_stream) return;
  cudaEventRecord(h->ev_join, 0);
  cudaStreamWaitEvent(h->stream, h->ev_join, 0);
}

cudaError_t copy_in(fredopt_t h, void* dst, const void* src, size_t bytes, uint32_t flags) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, dev_ptr(flags) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         h->stream);
}
cudaError_t copy_out(fredopt_t h, void* dst, const void* src, size_t bytes, uint32_t flags) {
  if (bytes == 0 || !dst) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, dev_ptr(flags) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         h->stream);
}

// Balanced contiguous split of rows [0, n_rows) into `parts` ranges by
// cost(row) = nnz(row) + row_cost.  Returns parts+1 boundaries.
std::vector<int64_t> partition_rows(const std::vector<int64_t>& rp, int64_t n_rows, int parts,
                                    int64_t row_cost) {
  std::vector<int64_t> b(parts + 1, n_rows);
  b[0] = 0;
  const double total = (double)(rp[n_rows] - rp[0]) + (double)row_cost * (double)n_rows;
  int64_t lo = 0;
  for (int k = 1; k < parts; ++k) {
    const double target = total * k / parts;
    int64_t a = lo, z = n_rows;  // first r with prefix(r) >= target
    while (a < z) {
      const int64_t m = (a + z) / 2;
      const double pre = (double)(rp[m] - rp[0]) + (double)row_cost * (double)m;
      if (pre < target) a = m + 1;
      else z = m;
    }
    b[k] = a;
    lo = a;
  }
  return b;
}

// Row ranges [r0, r1) for `parts` warps over the union of the row ranges
// `ranges` (each split in nnz-balanced contiguous pieces; warps are shared
// among ranges in proportion to their cost).  Returns 2*parts values.
std::vector<int64_t> partition_pairs(const std::vector<int64_t>& rp,
                                     const std::vector<std::pair<int64_t, int64_t>>& ranges, int parts,
                                     int64_t row_cost) {
  std::vector<int64_t> out(2 * (size_t)parts, 0);
  std::vector<size_t> live;
  double total = 0.0;
  std::vector<double> cost(ranges.size(), 0.0);
  for (size_t k = 0; k < ranges.size(); ++k) {
    const int64_t a = ranges[k].first, z = ranges[k].second;
    if (z <= a) continue;
    cost[k] = (double)(rp[z] - rp[a]) + (double)row_cost * (double)(z - a);
    total += cost[k];
    live.push_back(k);
  }
  int used = 0;
  for (size_t i = 0; i < live.size(); ++i) {
    const size_t k = live[i];
    const int later = (int)(live.size() - 1 - i);
    int w;
    if (later == 0) {
      w = parts - used;
    } else {
      w = (int)std::llround(parts * (total > 0 ? cost[k] / total : 0.0));
      w = std::max(1, std::min(w, parts - used - later));
    }
    if (w <= 0) break;
    const int64_t a = ranges[k].first, z = ranges[k].second;
    const double tot = cost[k];
    int64_t lo = a;
    for (int j = 0; j < w; ++j) {
      int64_t x = z;
      if (j + 1 < w) {
        const double target = tot * (j + 1) / w;
        int64_t y = z;
        x = lo;
        while (x < y) {  // first row m with prefix(m) >= target
          const int64_t m = (x + y) / 2;
          const double pre = (double)(rp[m] - rp[a]) + (double)row_cost * (double)(m - a);
          if (pre < target) x = m + 1;
          else y = m;
        }
      }
      out[2 * (used + j)] = lo;
      out[2 * (used + j) + 1] = x;
      lo = x;
    }
    used += w;
  }
  return out;
}

template <typename T>
cudaError_t upload_vec(fredopt_t h, DBuf<T>& d, const std::vector<T>& v) {
  cudaError_t e = d.alloc(v.size());
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream);
}

int value_bytes(int fmt) { return fmt == FREDOPT_FP32 ? 4 : 2; }

void free_graph(fredopt_t h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->graph_nodes = 0;
  h->graph_timed = false;
  h->gtimers.clear();
}

// ---- timed launch helper ----
Timer& next_timer(fredopt_t h, int cls) {
  if (h->timers_used == h->timers.size()) {
    Timer t;
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    h->timers.push_back(t);
  }
  Timer& t = h->timers[h->timers_used++];
  t.cls = cls;
  return t;
}

template <class F>
void run(fredopt_t h, int cls, F&& f) {
  if (h->timing) {
    Timer& t = next_timer(h, cls);
    // under stream capture the external flag makes each record a graph node;
    // every replay points those nodes at fresh events (fredopt_iterate)
    const unsigned fl = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaEventRecordWithFlags(t.a, h->stream, fl);
    f();
    cudaEventRecordWithFlags(t.b, h->stream, fl);
  } else {
    f();
  }
  h->launches += 1;
}

void collect_timers(fredopt_t h) {
  if (!h->timers_used) return;
  cudaStreamSynchronize(h->stream);
  for (size_t i = 0; i < h->timers_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->timers[i].a, h->timers[i].b) == cudaSuccess) {
      h->kms[h->timers[i].cls] += ms;
      h->klaunch[h->timers[i].cls] += 1;
    }
  }
  h->timers_used = 0;
}

// Claimed tiles pay off when a pass is long enough for the SMs' different
// streaming rates to matter; below kClaimMinNnzPerWarp nonzeros per warp the
// claims cost more than they balance (tile_balance 2 claims always).
constexpr int64_t kClaimMinNnzPerWarp = 16384;
bool claim_tiles(fredopt_t h) {
  if (h->prm.tile_balance == 2) return true;
  return h->prm.tile_balance == 1 && h->nnz_hot >= kClaimMinNnzPerWarp * (int64_t)h->geo.fwd_warps;
}

FwdArgs fwd_args(fredopt_t h, bool hot) {
  FwdArgs a{};
  a.rp = h->rp.p;
  a.col = h->col.p;
  a.col16 = h->col16.p;
  a.n_elems = (int64_t)(h->col16.p ? h->col16.n : h->col.n);
  a.Dv = h->Dv.p;
  a.Lv = h->Lv.p;
  a.sD = h->fmt ? h->sD.p : nullptr;
  a.sL = h->fmt ? h->sL.p : nullptr;
  a.warp_row = hot ? h->warp_row_hot.p : h->warp_row_all.p;
  if (hot && claim_tiles(h) && h->n_tiles_hot > 0) {
    a.warp_row = h->tile_row_hot.p;
    a.sched = h->fsched.p;
  }
  a.n_x = h->n;
  a.n_x_pad = h->n_pad;
  a.mask = h->mask.p;
  a.n_hot = h->n_hot;
  a.n_warps = a.sched ? h->n_tiles_hot : h->geo.fwd_warps;
  a.st = h->st.p;
  a.voxel = h->perm ? h->voxel.p : nullptr;
  return a;
}

BwdArgs bwd_args(fredopt_t h, const float2* coef) {
  BwdArgs b{};
  b.st = h->st.p;
  b.n_rows = h->n_hot;
  b.n_elems = (int64_t)h->crow.n;
  b.n_ovf = (int32_t)h->n_wide_blocks;
  b.row = h->crow.p;
  b.row16 = h->crow16.p;
  b.hdr = h->chdr.p;
  b.ovf = h->covf.p;
  b.Dv = h->DTv.p;
  b.Lv = h->LTv.p;
  b.chunk_ptr = h->chunk_ptr.p;
  b.warp_chunk = h->warp_chunk.p;
  b.coef = coef;
  b.chunk_sum = h->chunk_sum.p;
  b.n_warps = h->geo.bwd_warps;
  if (claim_tiles(h) && h->n_tiles_bwd > 0) {
    b.warp_chunk = h->tile_chunk.p;
    b.n_warps = h->n_tiles_bwd;
    b.sched = h->bsched.p;
  }
  return b;
}

ColArgs col_args(fredopt_t h) {
  ColArgs c{};
  c.col_chunk = h->col_chunk.p;
  c.chunk_sum = h->chunk_sum.p;
  c.n = h->n;
  c.k2part = h->part.p + h->off_k2;
  c.k2_blocks = h->geo.row_blocks;
  c.W_all = h->W_all;
  c.st = h->st.p;
  c.log = h->log.p;
  c.use_u = 1;
  return c;
}

ConArgs con_args(fredopt_t h) {
  ConArgs c{};
  c.yw = h->yw.p;
  c.mask = h->mask.p;
  c.dd = h->mdd.p;
  c.ll = h->mll.p;
  c.dl = h->mdl.p;
  c.sD = h->fmt ? h->sD.p : nullptr;
  c.sL = h->fmt ? h->sL.p : nullptr;
  c.n_hot = h->n_hot;
  c.rows = h->con_rows.p;
  c.n_list = h->n_con_rows;
  c.gam = h->gam.p;
  c.part = h->part.p + h->off_k2;
  c.st = h->st.p;
  return c;
}


// Blocks of the block-iterative sweep: the streamed rows with nonzeros that
// lie in some structure, in device (= ascending voxel) order, cut into groups
// of S = ceil(count / m) rows; block t covers the device rows from its first
// structure row to the next block's first.  Builds each block's forward
// schedule and the CSC position table of the block boundaries.
int build_sweep(fredopt_t h, int m) {
  if (h->sweep_m == m) return FREDOPT_OK;
  cudaStream_t s = h->stream;
  std::vector<int64_t> C;
  for (int64_t r = 0; r < h->n_hot_ne; ++r)
    if (h->h_mask[r] != 0) C.push_back(r);
  h->h_sweep_bounds.clear();
  h->sweep_wr_off.clear();
  h->sweep_warps.clear();
  h->sweep_nb = 0;
  if (!C.empty()) {
    const int64_t S = ((int64_t)C.size() + m - 1) / m;
    const int nb = (int)(((int64_t)C.size() + S - 1) / S);
    for (int t = 0; t < nb; ++t) h->h_sweep_bounds.push_back(C[(size_t)t * S]);
    h->h_sweep_bounds.push_back(C.back() + 1);
    h->sweep_nb = nb;
  }
  std::vector<int64_t> wr;
  for (int t = 0; t < h->sweep_nb; ++t) {
    const int64_t r0 = h->h_sweep_bounds[t], r1 = h->h_sweep_bounds[t + 1];
    const int warps = (int)std::max<int64_t>(1, std::min<int64_t>(h->geo.fwd_warps, r1 - r0));
    const std::vector<int64_t> p = partition_pairs(h->h_rp, {{r0, r1}}, warps, h->row_cost);
    h->sweep_wr_off.push_back((int64_t)wr.size() / 2);
    h->sweep_warps.push_back(warps);
    wr.insert(wr.end(), p.begin(), p.end());
  }
  if (wr.empty()) wr.assign(2, 0);
  CK(upload_vec(h, h->sweep_wr, wr));
  const int nbnd = h->sweep_nb + 1;
  std::vector<int64_t> bnd = h->h_sweep_bounds;
  if (bnd.empty()) bnd.assign(1, 0);
  CK(upload_vec(h, h->sweep_bounds_d, bnd));
  CK(h->sweep_pos.alloc((size_t)std::max(1, nbnd) * h->n));
  if (h->sweep_nb > 0) launch_sweep_pos(h->cp.p, h->crow.p, h->n, h->sweep_bounds_d.p, nbnd, h->sweep_pos.p, s);
  CK(h->xs.ensure(h->n_pad));
  CK(cudaMemsetAsync(h->xs.p, 0, h->n_pad * sizeof(float), s));
  CK(h->ys.ensure(std::max<int64_t>(1, h->n_hot)));
  CK(cudaMemsetAsync(h->ys.p, 0, std::max<int64_t>(1, h->n_hot) * sizeof(float2), s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  h->sweep_m = m;
  return FREDOPT_OK;
}

// One block-iterative sweep from x = w + coef * g (use_coef) or x = w, into out.
void enqueue_sweep(fredopt_t h, const float* w, int use_coef, double lam, double prio_scale, int norm,
                   int in_solve, float* out) {
  const Geometry& G = h->geo;
  cudaStream_t s = h->stream;
  run(h, 5, [&] { launch_sweep_start(h->n, w, h->g.p, use_coef, h->xs.p, h->st.p, s); });
  for (int t = 0; t < h->sweep_nb; ++t) {
    FwdArgs fa = fwd_args(h, true);
    fa.warp_row = h->sweep_wr.p + 2 * h->sweep_wr_off[t];
    fa.n_warps = h->sweep_warps[t];
    fa.sched = nullptr;  // the block's own static tiles
    fa.x = h->xs.p;
    fa.y = h->ys.p;
    run(h, 0, [&] { launch_forward(G, h->fmt, EPI_STORE, h->hint_fwd, fa, h->tab, s); });
    ConArgs k2 = con_args(h);
    k2.yw = h->ys.p;
    k2.yg = nullptr;
    k2.use_coef = 0;
    k2.rows = nullptr;  // the block's row range
    k2.r0 = h->h_sweep_bounds[t];
    k2.n_hot = h->h_sweep_bounds[t + 1];
    // one CTA per 256 rows of the block, at most the usual grid
    const int k2_grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(G.row_blocks, (k2.n_hot - k2.r0 + 255) / 256));
    run(h, 2, [&] { launch_constraints(G, h->tab, k2, s, k2_grid); });
    SweepArgs sa{};
    sa.pos0 = h->sweep_pos.p + (size_t)t * h->n;
    sa.pos1 = h->sweep_pos.p + (size_t)(t + 1) * h->n;
    sa.row = h->crow.p;
    sa.Dv = h->DTv.p;
    sa.Lv = h->LTv.p;
    sa.gam = h->gam.p;
    sa.x = h->xs.p;
    sa.n = h->n;
    sa.k2part = h->part.p + h->off_k2;
    sa.k2_blocks = k2_grid;
    sa.norm = norm;
    sa.lam = lam;
    sa.prio_scale = prio_scale;
    sa.in_solve = in_solve;
    sa.st = h->st.p;
    run(h, 1, [&] { launch_sweep_update(G, h->fmt, sa, s); });
  }
  run(h, 3, [&] { launch_sweep_finish(G, h->n, h->xs.p, out, in_solve, h->st.p, h->log.p, s); });
}

// One superiorized iteration (Fig. 3 around the simultaneous Fig. 2).
void enqueue_iteration(fredopt_t h) {
  const Geometry& G = h->geo;
  const Tables& t = h->tab;
  cudaStream_t s = h->stream;
  const int N = h->prm.reductions;
  const bool pert = N > 0 && t.n_obj > 0;
  double* part_f = h->part.p + h->off_f;
  double* part_bc = h->part.p + h->off_bc;
  double* part_g = h->part.p + h->off_g;
  FwdArgs fa = fwd_args(h, true);
  fa.x = h->w.p;
  fa.y = h->yw.p;
  if (pert) {
    fa.r_out = h->r.p;
    fa.part = part_f;
    run(h, 0, [&] { launch_forward(G, h->fmt, EPI_OBJ, h->hint_fwd, fa, t, s); });
    for (int step = 0; step < N; ++step) {
      int nf = fa.n_warps;
      if (step > 0) {
        run(h, 5, [&] { launch_apply_step(h->n_hot, h->n, h->w.p, h->g.p, h->yw.p, h->yg.p, h->st.p, s); });
        run(h, 5, [&] {
          launch_row_objective(G, t, h->yw.p, h->mask.p, fa.sD, fa.sL, h->n_hot, h->r.p, part_f, s);
        });
        nf = G.row_blocks;
      }
      BwdArgs ba = bwd_args(h, h->r.p);
      run(h, 1, [&] { launch_backward(G, h->fmt, h->hint_bwd, h->obj_dose, ba, s); });
      ColArgs ca = col_args(h);
      ca.out = h->g.p;
      ca.part = part_g;
      run(h, 3, [&] { launch_colfinish(G, COL_GRAD, ca, s); });
      FwdArgs fb = fa;
      fb.x = h->g.p;
      fb.y = h->yg.p;
      fb.r_in = h->r.p;
      fb.r_out = nullptr;
      fb.part = part_bc;
      run(h, 0, [&] { launch_forward(G, h->fmt, EPI_BC, h->hint_fwd, fb, t, s); });
      run(h, 4, [&] {
        launch_finish(step, part_f, nf, part_bc, fa.n_warps, part_g, G.col_blocks, h->st.p,
                      h->part.p + h->off_stage, h->part.p + h->off_btab, kBetaTable, s);
      });
    }
  } else {
    run(h, 0, [&] { launch_forward(G, h->fmt, EPI_STORE, h->hint_fwd, fa, t, s); });
  }
  if (h->prm.sweep_blocks > 0 && t.n_con > 0) {
    enqueue_sweep(h, h->w.p, pert ? 1 : 0, h->lam, 1.0, h->prm.cimmino_norm, 1, h->w.p);
    return;
  }
  ConArgs k2 = con_args(h);
  k2.yg = pert ? h->yg.p : nullptr;
  k2.use_coef = pert ? 1 : 0;
  run(h, 2, [&] { launch_constraints(G, t, k2, s); });
  if (t.n_con > 0) {
    BwdArgs bb = bwd_args(h, h->gam.p);
    run(h, 1, [&] { launch_backward(G, h->fmt, h->hint_bwd, true, bb, s); });
  }
  ColArgs cc = col_args(h);
  cc.w = h->w.p;
  cc.g = h->g.p;
  cc.use_coef = pert ? 1 : 0;
  cc.use_u = t.n_con > 0 ? 1 : 0;
  cc.norm = h->prm.cimmino_norm;
  cc.lam = h->lam;
  cc.in_solve = 1;
  // norm ALL without decay: the scale lam eta^k / W_all is fixed (the same
  // FP64 operations the kernel would do)
  cc.has_scale = (cc.norm != FREDOPT_NORM_VIOLATED && h->prm.eta == 1.0) ? 1 : 0;
  cc.scale = h->W_all > 0.0 ? cc.lam * 1.0 / h->W_all : 0.0;
  cc.log_block = cc.has_scale;
  run(h, 3, [&] { launch_colfinish(G, COL_PROJ, cc, s); });
}

// Tiles for warps that claim them in order (guided self-scheduling): the
// first W tiles each hold half of a warp's share of rows [0, n) (cost:
// nonzeros + row_cost per row), the next W a quarter, then an eighth, a
// sixteenth, a thirty-second, and 2W tiles of a sixty-fourth, so the last
// tiles to be claimed are short and the warps finish close together.
// Always kGuidedTilesPerWarp * W tiles (some may be empty), so the tile
// count, which kernels and captured graphs hold by value, does not depend on
// row_cost.  Returns 2 * count row bounds.
constexpr int kGuidedTilesPerWarp = 7;
std::vector<int64_t> guided_tiles(const std::vector<int64_t>& rp, int64_t n, int W, int64_t row_cost) {
  const int count = kGuidedTilesPerWarp * W;
  std::vector<int64_t> out(2 * (size_t)count, n > 0 ? n : 0);
  if (n <= 0 || W <= 0) return out;
  auto prefix = [&](int64_t r) { return (double)(rp[r] - rp[0]) + (double)row_cost * (double)r; };
  const double share = prefix(n) / W;
  const std::pair<double, int> rounds[] = {{0.5, W}, {0.25, W}, {0.125, W}, {0.0625, W}, {0.03125, W},
                                           {0.015625, 2 * W}};
  double target = 0.0;
  int64_t lo = 0;
  int k = 0;
  for (const auto& rd : rounds) {
    for (int i = 0; i < rd.second; ++i, ++k) {
      target += rd.first * share;
      int64_t hi = n;
      if (k + 1 < count) {
        int64_t x = lo, y = n;  // first row m with prefix(m) >= target
        while (x < y) {
          const int64_t m = (x + y) / 2;
          if (prefix(m) < target) x = m + 1;
          else y = m;
        }
        hi = x;
      }
      out[2 * (size_t)k] = lo;
      out[2 * (size_t)k + 1] = hi;
      lo = hi;
    }
  }
  return out;
}

// Warp partitions.  A segment's sum does not depend on which warp streams it
// (lanes take elements by their absolute block-aligned position and add them
// in order), so these weights change the speed, never a result bit.
int set_fwd_schedule(fredopt_t h, int64_t row_cost) {
  const std::vector<int64_t> wr = partition_pairs(h->h_rp, {{0, h->n_hot_ne}}, h->geo.fwd_warps, row_cost);
  const std::vector<int64_t> wa = partition_pairs(
      h->h_rp, {{0, h->n_hot_ne}, {h->n_hot, h->n_hot + h->n_cold_ne}}, h->geo.fwd_warps, row_cost);
  CK(cudaMemcpyAsync(h->warp_row_hot.p, wr.data(), wr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->warp_row_all.p, wa.data(), wa.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  const std::vector<int64_t> tl = guided_tiles(h->h_rp, h->n_hot_ne, h->geo.fwd_warps, row_cost);
  if ((size_t)h->tile_row_hot.n < std::max<size_t>(2, tl.size())) CK(h->tile_row_hot.alloc(std::max<size_t>(2, tl.size())));
  if (!tl.empty())
    CK(cudaMemcpyAsync(h->tile_row_hot.p, tl.data(), tl.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->n_tiles_hot = (int)(tl.size() / 2);
  h->row_cost = row_cost;
  return FREDOPT_OK;
}

int set_bwd_schedule(fredopt_t h, int64_t chunk_cost) {
  const std::vector<int64_t> w64 = partition_rows(h->h_cptr, h->n_chunks, h->geo.bwd_warps, chunk_cost);
  const std::vector<int32_t> w32(w64.begin(), w64.end());
  CK(cudaMemcpyAsync(h->warp_chunk.p, w32.data(), w32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  // claimed tiles: guided sizes over the chunks (the same rule as the forward rows)
  const std::vector<int64_t> tl = guided_tiles(h->h_cptr, h->n_chunks, h->geo.bwd_warps, chunk_cost);
  std::vector<int32_t> tb(tl.size() / 2 + 1, 0);
  for (size_t k = 0; k < tl.size() / 2; ++k) tb[k] = (int32_t)tl[2 * k];
  tb.back() = tl.empty() ? 0 : (int32_t)tl.back();
  if ((size_t)h->tile_chunk.n < tb.size()) CK(h->tile_chunk.alloc(tb.size()));
  CK(cudaMemcpyAsync(h->tile_chunk.p, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->n_tiles_bwd = (int)(tb.size() - 1);
  h->chunk_cost = chunk_cost;
  return FREDOPT_OK;
}

// Objective (Eq. 2 terms) of the streamed rows without nonzeros: their dose
// and LET-weighted dose are 0 for every w, so each term contributes w*T^2.
double f_empty(fredopt_t h) {
  double f = 0.0;
  for (int64_t r = h->n_hot_ne; r < h->n_hot; ++r) {
    const uint32_t m = h->h_mask[r];
    if (!m) continue;
    for (int i = 0; i < h->tab.n_obj; ++i)
      if ((m >> h->tab.obj[i].bit) & 1u) f += h->tab.obj[i].weight * h->tab.obj[i].target * h->tab.obj[i].target;
  }
  return f;
}

int need_loaded(fredopt_t h) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  if (!h->loaded) return fail(h, FREDOPT_ERR_NOT_LOADED, "no influence matrices loaded");
  return FREDOPT_OK;
}

// Upload a spot vector (n floats) into a padded device buffer.
int load_spot_vec(fredopt_t h, DBuf<float>& dst, const float* src, uint32_t flags) {
  CK(copy_in(h, dst.p, src, (size_t)h->n * sizeof(float), flags));
  return FREDOPT_OK;
}

int check_sticky(fredopt_t h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  int err = 0;
  CK(cudaMemcpy(&err, &h->st.p->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    const int zero = 0;
    cudaMemcpy(&h->st.p->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
    // a pass that gave up may have left its tile counters set
    if (h->fsched.p) cudaMemset(h->fsched.p, 0, 2 * sizeof(unsigned int));
    if (h->bsched.p) cudaMemset(h->bsched.p, 0, 2 * sizeof(unsigned int));
    if (err & 2) return fail(h, FREDOPT_ERR_PATTERN, "checked build: an index or tile range out of bounds");
    return fail(h, FREDOPT_ERR_TIMEOUT, "a bounded device-side wait gave up (bulk copy)");
  }
  return FREDOPT_OK;
}

// FP64 pass of every row for w (host or device per flags; null = the current
// iterate of a begun solve) into y64, as in fredopt_end.
int final_pass_y64(fredopt_t h, const float* w, uint32_t flags) {
  cudaStream_t s = h->stream;
  const float* x = nullptr;
  if (w) {
    int rc = load_spot_vec(h, h->xbuf, w, flags);
    if (rc) return rc;
    x = h->xbuf.p;
  } else {
    if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "w is null and no solve is begun");
    x = h->w.p;
  }
  CK(h->y64.ensure(std::max<int64_t>(1, h->V)));
  CK(cudaMemsetAsync(h->y64.p, 0, std::max<int64_t>(1, h->V) * sizeof(double2), s));
  FwdArgs fa = fwd_args(h, false);
  fa.x = x;
  fa.y64 = h->y64.p;
  fa.dose_out = nullptr;
  fa.letd_out = nullptr;
  run(h, 0, [&] { launch_forward(h->geo, h->fmt, EPI_FINAL, false, fa, h->tab, s); });
  CK(cudaGetLastError());
  return FREDOPT_OK;
}

// Rank k (1 = largest) of the value received by the fraction `frac` of n
// voxels: ceil(frac * n), a product within 1e-9 * max(1, product) of an
// integer counting as that integer, kept in [1, n].
int64_t at_volume_rank(double frac, int64_t n) {
  volatile double t = frac * (double)n;  // rounded product (never fused with what follows)
  const double tv = t;
  const double r = std::floor(tv + 0.5);
  const double k = (std::fabs(tv - r) <= 1e-9 * std::max(1.0, tv)) ? r : std::ceil(tv);
  return std::min<int64_t>(std::max<int64_t>((int64_t)k, 1), n);
}

float key_to_float(uint32_t key) {
  const uint32_t u = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
  float f;
  std::memcpy(&f, &u, sizeof(f));
  return f;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// =================================================================== ABI

extern "C" {

void fredopt_default_params(fredopt_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->beta0 = -1.0;
  p->eta = 1.0;
  p->reductions = 1;
  p->max_trials = 50;
  p->cimmino_norm = FREDOPT_NORM_ALL;
  p->grad_normalize = 1;
  p->c_cdl = 0.04;
  p->log_capacity = 4096;
  p->use_graphs = 1;
  p->tile_balance = 1;
}

const char* fredopt_strerror(int code) {
  const int i = -code;
  if (i < 0 || i >= (int)(sizeof(kErrNames) / sizeof(kErrNames[0]))) return "unknown error";
  return kErrNames[i];
}

const char* fredopt_last_error(fredopt_t h) { return h ? h->last_error.c_str() : "null handle"; }

int fredopt_create(fredopt_t* out, int device, void* cuda_stream) {
  if (!out) return FREDOPT_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return FREDOPT_ERR_INVALID_ARG;
  }
  fredopt_ctx* h = new fredopt_ctx();
  h->device = device;
  DeviceGuard dg(device);
  if (init_kernels(&h->geo_full, device) != 0) {
    delete h;
    cudaGetLastError();
    return FREDOPT_ERR_CUDA;
  }
  h->geo = h->geo_full;
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  h->l2_bytes = (size_t)l2;
  if (cuda_stream) {
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return FREDOPT_ERR_CUDA;
    }
    h->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&h->ev_it0) != cudaSuccess || cudaEventCreate(&h->ev_it1) != cudaSuccess ||
      h->st.alloc(1) != cudaSuccess || h->errw.alloc(1) != cudaSuccess) {
    fredopt_destroy(h);
    return FREDOPT_ERR_CUDA;
  }
  cudaMemsetAsync(h->st.p, 0, sizeof(DevState), h->stream);
  fredopt_default_params(&h->prm);
  h->tab.c = 0.04;
  cudaStreamSynchronize(h->stream);
  *out = h;
  return FREDOPT_OK;
}

int fredopt_destroy(fredopt_t h) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_graph(h);
  for (auto& t : h->timers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_it0) cudaEventDestroy(h->ev_it0);
  if (h->ev_it1) cudaEventDestroy(h->ev_it1);
  cudaStream_t own = h->own_stream ? h->stream : nullptr;
  delete h;  // frees every device buffer
  if (own) cudaStreamDestroy(own);
  return FREDOPT_OK;
}

int fredopt_load_influence(fredopt_t h, int64_t n_vox, int32_t n_spots, int64_t nnz,
                           const int64_t* row_ptr, const int32_t* col, const float* D_val,
                           const float* L_val, const uint32_t* voxel_mask, int format,
                           uint32_t flags) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  const int fmt = format & 0xff;
  const bool roi = (format & FREDOPT_ROWS_ROI) != 0;
  if (fmt < 0 || fmt > 2 || (format & ~0x7ff))
    return fail(h, FREDOPT_ERR_INVALID_ARG, "format must be FP32/BF16/FP16 | ROWS_ALL/ROI | INDEX32 | SHARED");
  if (n_vox < 0 || n_spots < 1 || nnz < 0 || nnz > 2147483647LL || n_vox > 2147483647LL)
    return fail(h, FREDOPT_ERR_SHAPE, "need n_vox >= 0, n_spots >= 1, 0 <= nnz < 2^31");
  if (!row_ptr || !voxel_mask || (nnz > 0 && (!col || !D_val || !L_val)))
    return fail(h, FREDOPT_ERR_INVALID_ARG, "null array");
  DeviceGuard dg(h->device);
  free_graph(h);
  h->loaded = false;
  h->begun = false;
  h->sweep_m = 0;
  int rc = FREDOPT_OK;
  cudaStream_t s = h->stream;
  join_in(h);

  // every index / value array is zero padded past its last nonzero
  const int64_t nnz_alloc = ((nnz + 255) & ~255LL) + kPadElems;

  // ---- host inputs: their upload is issued first, so that the copy engine
  // runs while the host checks row_ptr and orders the rows
  DBuf<int32_t> col_in;
  DBuf<float> D_in, L_in;
  const int32_t* colp = col;
  const float *Dp = D_val, *Lp = L_val;
  if (!dev_ptr(flags)) {
    CK(col_in.alloc(nnz_alloc));
    CK(D_in.alloc(nnz_alloc));
    CK(L_in.alloc(nnz_alloc));
    CK(cudaMemsetAsync(col_in.p + nnz, 0, (nnz_alloc - nnz) * sizeof(int32_t), s));
    CK(cudaMemsetAsync(D_in.p + nnz, 0, (nnz_alloc - nnz) * sizeof(float), s));
    CK(cudaMemsetAsync(L_in.p + nnz, 0, (nnz_alloc - nnz) * sizeof(float), s));
    if (nnz) {
      CK(cudaMemcpyAsync(col_in.p, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(D_in.p, D_val, nnz * sizeof(float), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(L_in.p, L_val, nnz * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    colp = col_in.p;
    Dp = D_in.p;
    Lp = L_in.p;
  }

  // ---- row_ptr and the mask on the host (read in place when they are host
  // memory); row_ptr checked on the host
  std::vector<int64_t> rp_copy;
  std::vector<uint32_t> m_copy;
  const int64_t* rp0 = row_ptr;
  const uint32_t* m0 = voxel_mask;
  if (dev_ptr(flags)) {
    rp_copy.resize(n_vox + 1);
    m_copy.resize(n_vox);
    CK(cudaMemcpyAsync(rp_copy.data(), row_ptr, (n_vox + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (n_vox) CK(cudaMemcpyAsync(m_copy.data(), voxel_mask, n_vox * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rp0 = rp_copy.data();
    m0 = m_copy.data();
  }
  if (rp0[0] != 0 || rp0[n_vox] != nnz) return fail(h, FREDOPT_ERR_PATTERN, "row_ptr[0] != 0 or row_ptr[n_vox] != nnz");
  for (int64_t i = 0; i < n_vox; ++i)
    if (rp0[i + 1] < rp0[i]) return fail(h, FREDOPT_ERR_PATTERN, "row_ptr not monotone");

  // ---- device order of rows: streamed rows with nonzeros, streamed rows
  // without, other rows with nonzeros, other rows without (each ascending);
  // one pass over row_ptr and the mask assigns the groups
  std::vector<uint8_t> grp(n_vox);
  int64_t c0 = 0, c1 = 0, c2 = 0;  // counts in locals: no store-to-load chain between rows
  for (int64_t i = 0; i < n_vox; ++i) {
    const int g = ((!roi || m0[i] != 0) ? 0 : 2) + (rp0[i + 1] > rp0[i] ? 0 : 1);
    grp[i] = (uint8_t)g;
    c0 += g == 0;
    c1 += g == 1;
    c2 += g == 2;
  }
  const int64_t n_hot_ne = c0;
  const int64_t n_hot = c0 + c1;
  const int64_t n_cold_ne = c2;
  std::vector<int64_t> order(n_vox);
  bool perm = false;
  {
    int64_t p0 = 0, p1 = c0, p2 = c0 + c1, p3 = c0 + c1 + c2;
    for (int64_t i = 0; i < n_vox; ++i) {
      int64_t r;
      switch (grp[i]) {
        case 0: r = p0++; break;
        case 1: r = p1++; break;
        case 2: r = p2++; break;
        default: r = p3++; break;
      }
      order[r] = i;
      perm |= r != i;
    }
  }
  std::vector<int64_t> rpd(n_vox + 1);
  if (perm) {
    rpd[0] = 0;
    for (int64_t r = 0; r < n_vox; ++r) rpd[r + 1] = rpd[r] + (rp0[order[r] + 1] - rp0[order[r]]);
  } else {
    std::memcpy(rpd.data(), rp0, (n_vox + 1) * sizeof(int64_t));
  }

  // ---- validate (on the input layout)
  DBuf<int64_t> rp_in;
  CK(rp_in.alloc(n_vox + 1));
  CK(cudaMemcpyAsync(rp_in.p, rp0, (n_vox + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(h->errw.p, 0, sizeof(int), s));
  launch_validate(rp_in.p, colp, Dp, Lp, n_vox, n_spots, nnz, h->errw.p, s);
  CK(cudaGetLastError());
  int verr = 0;
  CK(cudaMemcpyAsync(&verr, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (verr & 1) return fail(h, FREDOPT_ERR_PATTERN, "column index out of range or not strictly increasing within a row");
  if (verr & 2) return fail(h, FREDOPT_ERR_NONFINITE, "NaN or Inf in D or L");

  // ---- drop the previous plan
  h->rp.release(); h->col.release(); h->col16.release(); h->Dv.release(); h->Lv.release(); h->sD.release(); h->sL.release();
  h->voxel.release(); h->mask.release(); h->con_rows.release(); h->ucoef.release(); h->cp.release(); h->crow.release(); h->crow16.release(); h->chdr.release(); h->covf.release(); h->DTv.release(); h->LTv.release();

  // ---- FP32 CSR in device order (zero padded)
  DBuf<int32_t> col_d;
  DBuf<float> D_d, L_d;
  CK(upload_vec(h, h->rp, rpd));
  if (perm || dev_ptr(flags)) {
    CK(col_d.alloc(nnz_alloc));
    CK(D_d.alloc(nnz_alloc));
    CK(L_d.alloc(nnz_alloc));
    CK(cudaMemsetAsync(col_d.p + nnz, 0, (nnz_alloc - nnz) * sizeof(int32_t), s));
    CK(cudaMemsetAsync(D_d.p + nnz, 0, (nnz_alloc - nnz) * sizeof(float), s));
    CK(cudaMemsetAsync(L_d.p + nnz, 0, (nnz_alloc - nnz) * sizeof(float), s));
    if (perm) {
      // device row -> voxel: the gather's source rows, kept for the outputs
      CK(upload_vec(h, h->voxel, order));
      launch_gather_rows(rp_in.p, h->voxel.p, h->rp.p, n_vox, colp, Dp, Lp, col_d.p, D_d.p, L_d.p, s);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(s));
    } else if (nnz) {
      CK(cudaMemcpyAsync(col_d.p, col, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(D_d.p, D_val, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(L_d.p, L_val, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
  } else {
    std::swap(col_d.p, col_in.p); std::swap(col_d.n, col_in.n);
    std::swap(D_d.p, D_in.p); std::swap(D_d.n, D_in.n);
    std::swap(L_d.p, L_in.p); std::swap(L_d.n, L_in.n);
  }
  CK(cudaStreamSynchronize(s));
  col_in.release(); D_in.release(); L_in.release(); rp_in.release();
  std::swap(h->col.p, col_d.p); std::swap(h->col.n, col_d.n);

  // ---- value storage (quantised with power-of-two row scales, or FP32)
  if (fmt == FREDOPT_FP32) {
    h->Dv.p = reinterpret_cast<uint8_t*>(D_d.p); h->Dv.n = D_d.n * 4; D_d.p = nullptr; D_d.n = 0;
    h->Lv.p = reinterpret_cast<uint8_t*>(L_d.p); h->Lv.n = L_d.n * 4; L_d.p = nullptr; L_d.n = 0;
  } else {
    CK(h->Dv.alloc((size_t)nnz_alloc * 2));
    CK(h->Lv.alloc((size_t)nnz_alloc * 2));
    CK(cudaMemsetAsync(h->Dv.p, 0, (size_t)nnz_alloc * 2, s));
    CK(cudaMemsetAsync(h->Lv.p, 0, (size_t)nnz_alloc * 2, s));
    CK(h->sD.alloc(n_vox));
    CK(h->sL.alloc(n_vox));
    launch_quantize(fmt, h->rp.p, n_vox, D_d.p, L_d.p, h->Dv.p, h->Lv.p, h->sD.p, h->sL.p, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    D_d.release();
    L_d.release();
  }

  // ---- streamed rows: mask, FP64 moments
  h->V = n_vox; h->nnz = nnz; h->n = n_spots; h->n_pad = (n_spots + 3) & ~3;
  h->fmt = fmt; h->roi = roi; h->perm = perm; h->n_hot = n_hot; h->nnz_hot = rpd[n_hot];
  h->n_hot_ne = n_hot_ne; h->n_cold_ne = n_cold_ne;
  h->h_mask.resize(n_hot);
  for (int64_t r = 0; r < n_hot; ++r) h->h_mask[r] = m0[order[r]];
  if (perm) h->h_voxel = std::move(order);  // order is not used below
  else h->h_voxel.clear();
  CK(upload_vec(h, h->mask, h->h_mask));
  {
    // the constraint evaluation visits only these rows; the others' projection
    // coefficients stay 0
    std::vector<int64_t>& cr = h->h_con_rows;
    cr.clear();
    for (int64_t r = 0; r < n_hot; ++r)
      if (h->h_mask[r] != 0) cr.push_back(r);
    h->n_con_rows = (int64_t)cr.size();
    CK(upload_vec(h, h->con_rows, cr));
  }
  CK(h->mdd.alloc(n_hot)); CK(h->mll.alloc(n_hot)); CK(h->mdl.alloc(n_hot));
  CK(cudaMemsetAsync(h->mdd.p, 0, std::max<int64_t>(1, n_hot) * sizeof(double), s));
  CK(cudaMemsetAsync(h->mll.p, 0, std::max<int64_t>(1, n_hot) * sizeof(double), s));
  CK(cudaMemsetAsync(h->mdl.p, 0, std::max<int64_t>(1, n_hot) * sizeof(double), s));
  launch_moments(fmt, h->rp.p, n_hot_ne, h->Dv.p, h->Lv.p, fmt ? h->sD.p : nullptr, fmt ? h->sL.p : nullptr,
                 h->mdd.p, h->mll.p, h->mdl.p, s);
  CK(cudaGetLastError());

  // ---- launch shapes: the whole GPU, or with FREDOPT_SHARED one SM's
  // worth of CTAs per kSharedNnzPerSm nonzeros, so that the kernels of other
  // plans in a batch or on a server share the GPU (16 plans of 6e5-7e7
  // nonzeros, BF16, one batch graph: 13621 against 10560 plan-iterations/s;
  // 12831, 13205 and 12380 at 1e5, 2e5 and 8e5 nonzeros per SM)
  {
#ifndef FO_SHARED_NNZ_PER_SM
#define FO_SHARED_NNZ_PER_SM 400000
#endif
    constexpr int64_t kSharedNnzPerSm = FO_SHARED_NNZ_PER_SM;
    const Geometry& F = h->geo_full;
    int eff = F.n_sms;
    if (format & FREDOPT_SHARED)
      eff = (int)std::max<int64_t>(1, std::min<int64_t>(F.n_sms, (h->nnz_hot + kSharedNnzPerSm - 1) / kSharedNnzPerSm));
    Geometry g = F;
    g.n_sms = eff;
    g.fwd_blocks = F.fwd_blocks / F.n_sms * eff;
    g.fwd_warps = g.fwd_blocks * (g.fwd_threads / 32);
    g.bwd_blocks = F.bwd_blocks / F.n_sms * eff;
    g.bwd_warps = g.bwd_blocks * (g.bwd_threads / 32);
    g.row_blocks = F.row_blocks / F.n_sms * eff;
    g.col_blocks = F.col_blocks / F.n_sms * eff;
    h->geo = g;
  }

  // ---- CSC copy of the streamed rows (blocked stable counting transpose)
  {
    // rows without nonzeros (after the others in device order) add nothing
    // one wave of 1024-thread blocks over the whole GPU whatever the plan's
    // launch shapes (the transpose does not depend on its partition)
    const int n_blk = (int)std::max<int64_t>(1, std::min<int64_t>(h->geo_full.n_sms, n_hot_ne));
    std::vector<int64_t> blk = partition_rows(rpd, n_hot_ne, n_blk, 1);
    DBuf<int64_t> blk_d, tot_d;
    DBuf<int32_t> cnt;
    CK(upload_vec(h, blk_d, blk));
    CK(cnt.alloc((size_t)n_blk * n_spots));
    CK(cudaMemsetAsync(cnt.p, 0, (size_t)n_blk * n_spots * sizeof(int32_t), s));
    if (n_hot_ne > 0) launch_csc_count(h->rp.p, h->col.p, blk_d.p, n_blk, n_spots, cnt.p, s);
    CK(tot_d.alloc(n_spots));
    launch_csc_colsum(cnt.p, n_blk, n_spots, tot_d.p, s);
    CK(cudaGetLastError());
    std::vector<int64_t> tot(n_spots), cph(n_spots + 1);
    CK(cudaMemcpyAsync(tot.data(), tot_d.p, n_spots * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cph[0] = 0;
    for (int j = 0; j < n_spots; ++j) cph[j + 1] = cph[j] + tot[j];
    if (cph[n_spots] != h->nnz_hot) return fail(h, FREDOPT_ERR_CUDA, "CSC count mismatch");
    CK(upload_vec(h, h->cp, cph));
    launch_csc_offsets(cnt.p, n_blk, n_spots, h->cp.p, s);
    const int vb = value_bytes(fmt);
    const int64_t nh_alloc = ((h->nnz_hot + 255) & ~255LL) + kPadElems;
    CK(h->crow.alloc(nh_alloc));
    CK(h->DTv.alloc((size_t)nh_alloc * vb));
    CK(h->LTv.alloc((size_t)nh_alloc * vb));
    CK(cudaMemsetAsync(h->crow.p + h->nnz_hot, 0, (nh_alloc - h->nnz_hot) * sizeof(int32_t), s));
    CK(cudaMemsetAsync(h->DTv.p + (size_t)h->nnz_hot * vb, 0, (size_t)(nh_alloc - h->nnz_hot) * vb, s));
    CK(cudaMemsetAsync(h->LTv.p + (size_t)h->nnz_hot * vb, 0, (size_t)(nh_alloc - h->nnz_hot) * vb, s));
    CK(cudaMemsetAsync(h->errw.p, 0, sizeof(int), s));
    if (n_hot_ne > 0) {
      // scattered stores are limited by their count: one record per entry,
      // split into the three arrays by a coalesced pass (scratch freed here)
      DBuf<uint8_t> rec;
      const size_t rb = csc_fill_rec_bytes(h->geo, fmt, n_spots);
      if (rb) CK(rec.alloc((size_t)h->nnz_hot * rb));
      launch_csc_fill(h->geo, fmt, h->rp.p, h->col.p, h->Dv.p, h->Lv.p, blk_d.p, n_blk, n_spots, cnt.p,
                      h->crow.p, h->DTv.p, h->LTv.p, h->errw.p, rb ? rec.p : nullptr, h->nnz_hot, s);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(s));
    }
    CK(cudaGetLastError());
    int ferr = 0;
    CK(cudaMemcpyAsync(&ferr, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ferr) return fail(h, FREDOPT_ERR_TIMEOUT, "a bounded device-side wait gave up (CSC transpose)");

    // based 16-bit row indices for the transposed product (2 bytes less per
    // nonzero and pass; crow stays for the sweep and inspection)
    h->n_wide_blocks = 0;
    if (!(format & FREDOPT_INDEX32)) {
      const int64_t n_cblk = nh_alloc / 128;
      CK(h->crow16.alloc(nh_alloc));
      CK(h->chdr.alloc(n_cblk));
      CK(h->cnw.ensure(2));
      CK(cudaMemsetAsync(h->cnw.p, 0, 2 * sizeof(unsigned int), s));
      launch_narrow_rows(h->crow.p, n_cblk, h->crow16.p, h->chdr.p, h->cnw.p, s);
      CK(cudaGetLastError());
      unsigned int n_wide = 0;
      CK(cudaMemcpyAsync(&n_wide, h->cnw.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      CK(h->covf.alloc((size_t)std::max(1u, n_wide) * 128));
      launch_narrow_rows_wide(h->crow.p, n_cblk, h->chdr.p, h->covf.p, h->cnw.p + 1, n_wide, s);
      CK(cudaGetLastError());
      h->n_wide_blocks = n_wide;
    }

    // chunk schedule of the transposed product
    const int W3 = h->geo.bwd_warps;
    int64_t C = h->nnz_hot / ((int64_t)W3 * 8);
    C = std::max<int64_t>(256, std::min<int64_t>(8192, C));
    C = (C + 31) & ~31LL;
    std::vector<int64_t> cptr;
    std::vector<int32_t> cchunk(n_spots + 1);
    cptr.reserve(h->nnz_hot / C + n_spots + 1);
    for (int j = 0; j < n_spots; ++j) {
      cchunk[j] = (int32_t)cptr.size();
      for (int64_t p = cph[j]; p < cph[j + 1]; p += C) cptr.push_back(p);
    }
    cchunk[n_spots] = (int32_t)cptr.size();
    h->n_chunks = (int64_t)cptr.size();
    cptr.push_back(h->nnz_hot);
    CK(upload_vec(h, h->chunk_ptr, cptr));
    CK(upload_vec(h, h->col_chunk, cchunk));
    CK(cudaStreamSynchronize(s));
    h->h_cptr.swap(cptr);
    CK(h->warp_chunk.alloc(W3 + 1));
    rc = set_bwd_schedule(h, 16);
    if (rc) return rc;
  }

  // ---- 16-bit column indices for the forward stream: 2 bytes less per
  // nonzero, same sums.  Only with x staged in shared memory (that bounds
  // n_spots below 65536); the int32 copy served the CSC build and goes.
  if (!(format & FREDOPT_INDEX32) && n_spots <= 65536 && forward_uses_smem(h->geo, h->n_pad)) {
    CK(h->col16.alloc(h->col.n));
    launch_narrow_idx(h->col.p, h->col16.p, (int64_t)h->col.n, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    h->col.release();
  }

  // ---- row schedules of the forward product (rows with nonzeros only);
  // a row end (two warp reductions and bookkeeping) costs about as much as
  // streaming FO_ROW_COST nonzeros (fredopt_autotune can pick another weight)
#ifndef FO_ROW_COST
#define FO_ROW_COST 64
#endif
  h->h_rp = std::move(rpd);
  h->n_hot_ne = n_hot_ne;
  h->n_cold_ne = n_cold_ne;
  CK(h->warp_row_hot.alloc(2 * (size_t)h->geo.fwd_warps));
  CK(h->warp_row_all.alloc(2 * (size_t)h->geo.fwd_warps));
  CK(h->fsched.ensure(2));
  CK(cudaMemsetAsync(h->fsched.p, 0, 2 * sizeof(unsigned int), s));
  CK(h->bsched.ensure(2));
  CK(cudaMemsetAsync(h->bsched.p, 0, 2 * sizeof(unsigned int), s));
  rc = set_fwd_schedule(h, FO_ROW_COST);
  if (rc) return rc;
  // streaming (evict-first) loads when the streamed matrices do not fit in L2
  const double mat_bytes = (double)h->nnz_hot * ((h->col16.p ? 2.0 : 4.0) + 2.0 * value_bytes(fmt));
#ifndef FO_STREAM_HINT
#define FO_STREAM_HINT -1
#endif
  h->hint_fwd = FO_STREAM_HINT < 0 ? mat_bytes > 0.5 * (double)h->l2_bytes : FO_STREAM_HINT != 0;
  h->hint_bwd = h->hint_fwd;

  // ---- work buffers
  CK(h->w.alloc(h->n_pad)); CK(h->g.alloc(h->n_pad)); CK(h->xbuf.alloc(h->n_pad)); CK(h->gtmp.alloc(h->n_pad));
  CK(cudaMemsetAsync(h->w.p, 0, h->n_pad * sizeof(float), s));
  CK(cudaMemsetAsync(h->g.p, 0, h->n_pad * sizeof(float), s));
  CK(cudaMemsetAsync(h->xbuf.p, 0, h->n_pad * sizeof(float), s));
  CK(cudaMemsetAsync(h->gtmp.p, 0, h->n_pad * sizeof(float), s));
  CK(h->yw.alloc(n_hot)); CK(h->yg.alloc(n_hot)); CK(h->r.alloc(n_hot)); CK(h->gam.alloc(n_hot));
  // rows without nonzeros are never written by the forward product: keep them 0
  CK(cudaMemsetAsync(h->yw.p, 0, std::max<int64_t>(1, n_hot) * sizeof(float2), s));
  CK(cudaMemsetAsync(h->yg.p, 0, std::max<int64_t>(1, n_hot) * sizeof(float2), s));
  CK(cudaMemsetAsync(h->r.p, 0, std::max<int64_t>(1, n_hot) * sizeof(float2), s));
  // projection coefficients: rows without a structure bit are never written
  CK(cudaMemsetAsync(h->gam.p, 0, std::max<int64_t>(1, n_hot) * sizeof(float2), s));
  CK(h->chunk_sum.alloc(h->n_chunks));
  const Geometry& G = h->geo;
  // forward partials: one per tile (at most 7 guided tiles per warp)
  const int max_tiles = kGuidedTilesPerWarp * G.fwd_warps;
  h->off_f = 0;
  h->off_bc = h->off_f + std::max(max_tiles, G.row_blocks);
  h->off_g = h->off_bc + 2 * max_tiles;
  h->off_k2 = h->off_g + G.col_blocks;
  h->off_fin = h->off_k2 + 4 * G.row_blocks;
  h->off_cnt = h->off_fin + 8 * G.row_blocks;
  h->off_stage = h->off_cnt + 3 * G.row_blocks;
  h->off_btab = h->off_stage + 4 * kFinishBlocks;
  h->n_part = h->off_btab + kBetaTable;
  h->btab_alpha = -1.0;  // the table is refilled at the next fredopt_begin
  CK(h->part.alloc(h->n_part));
  CK(cudaMemsetAsync(h->part.p, 0, h->n_part * sizeof(double), s));
  h->y64.release(); h->yall.release(); h->fout_a.release(); h->fout_b.release();
  h->vin_a.release(); h->vin_b.release();
  CK(cudaStreamSynchronize(s));

  h->tab.n_con = 0;
  h->tab.n_obj = 0;
  h->have_con = false;
  h->obj_dose = false;
  h->W_all = 0.0;
  h->n_rows_reach = h->n_unreach = 0;
  h->loaded = true;
  return FREDOPT_OK;
}

int fredopt_set_constraints(fredopt_t h, int n, const fredopt_constraint* c) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (n < 0 || n > kMaxCon || (n > 0 && !c)) return fail(h, FREDOPT_ERR_INVALID_ARG, "0 <= n <= 32 constraints");
  for (int i = 0; i < n; ++i) {
    if (c[i].struct_bit >= 32 || c[i].kind < 0 || c[i].kind > 5 || !std::isfinite(c[i].bound) ||
        !(c[i].priority > 0.0) || !std::isfinite(c[i].priority))
      return fail(h, FREDOPT_ERR_INVALID_ARG, "constraint " + std::to_string(i) + " invalid");
  }
  DeviceGuard dg(h->device);
  free_graph(h);
  h->tab.n_con = n;
  for (int i = 0; i < n; ++i) {
    h->tab.con[i].bit = c[i].struct_bit;
    h->tab.con[i].kind = c[i].kind;
    h->tab.con[i].bound = c[i].bound;
    h->tab.con[i].prio = c[i].priority;
  }
  double* pc = h->part.p + h->off_cnt;
  launch_count_rows(h->geo, h->tab, h->mask.p, h->mdd.p, h->mll.p, h->mdl.p, h->n_hot, pc, h->stream);
  CK(cudaGetLastError());
  std::vector<double> hp(3 * h->geo.row_blocks);
  CK(cudaMemcpyAsync(hp.data(), pc, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  double nr = 0, nu = 0, W = 0;
  for (int b = 0; b < h->geo.row_blocks; ++b) {
    nr += hp[3 * b];
    nu += hp[3 * b + 1];
    W += hp[3 * b + 2];
  }
  h->n_rows_reach = (int64_t)nr;
  h->n_unreach = (int64_t)nu;
  h->W_all = W;
  h->have_con = true;
  return FREDOPT_OK;
}

int fredopt_set_objective(fredopt_t h, int n, const fredopt_objective_term* t) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (n < 0 || n > kMaxObj || (n > 0 && !t)) return fail(h, FREDOPT_ERR_INVALID_ARG, "0 <= n <= 32 terms");
  for (int i = 0; i < n; ++i)
    if (t[i].struct_bit >= 32 || (t[i].quantity != FREDOPT_Q_DOSE && t[i].quantity != FREDOPT_Q_CDL) ||
        !std::isfinite(t[i].target) || !(t[i].weight > 0.0) || !std::isfinite(t[i].weight))
      return fail(h, FREDOPT_ERR_INVALID_ARG, "objective term " + std::to_string(i) + " invalid");
  free_graph(h);
  h->tab.n_obj = n;
  h->obj_dose = false;
  for (int i = 0; i < n; ++i) {
    h->tab.obj[i].bit = t[i].struct_bit;
    h->tab.obj[i].q = t[i].quantity;
    h->tab.obj[i].target = t[i].target;
    h->tab.obj[i].weight = t[i].weight;
    if (t[i].quantity == FREDOPT_Q_DOSE) h->obj_dose = true;
  }
  if (h->begun) {
    DeviceGuard dg(h->device);
    h->st_host.f_empty = f_empty(h);
    CK(cudaMemcpyAsync(&h->st.p->f_empty, &h->st_host.f_empty, sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return FREDOPT_OK;
}

int fredopt_begin(fredopt_t h, const float* w0, double alpha, double relaxation,
                  const fredopt_params* params, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!w0) return fail(h, FREDOPT_ERR_INVALID_ARG, "w0 is null");
  fredopt_params p;
  if (params) p = *params;
  else fredopt_default_params(&p);
  if (!(alpha > 0.0 && alpha < 1.0)) return fail(h, FREDOPT_ERR_INVALID_ARG, "need 0 < alpha < 1");
  if (!(relaxation > 0.0 && relaxation <= 2.0)) return fail(h, FREDOPT_ERR_INVALID_ARG, "need 0 < relaxation <= 2");
  if (!(p.eta > 0.0 && p.eta <= 1.0)) return fail(h, FREDOPT_ERR_INVALID_ARG, "need 0 < eta <= 1");
  if (p.reductions < 0 || p.max_trials < 1 || p.log_capacity < 0 ||
      (p.cimmino_norm != FREDOPT_NORM_ALL && p.cimmino_norm != FREDOPT_NORM_VIOLATED) ||
      !(p.c_cdl > 0.0) || !std::isfinite(p.beta0) || p.sweep_blocks < 0 ||
      p.sweep_blocks > FREDOPT_MAX_SWEEP_BLOCKS || p.tile_balance < 0 || p.tile_balance > 2)
    return fail(h, FREDOPT_ERR_INVALID_ARG, "bad parameters");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  join_in(h);
  std::vector<float> hw(h->n);
  if (dev_ptr(flags)) {
    CK(cudaMemcpyAsync(hw.data(), w0, h->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else {
    std::memcpy(hw.data(), w0, h->n * sizeof(float));
  }
  double nrm = 0.0;
  for (float v : hw) {
    if (!std::isfinite(v)) return fail(h, FREDOPT_ERR_NONFINITE, "w0 not finite");
    if (v < 0.0f) return fail(h, FREDOPT_ERR_INVALID_ARG, "w0 must be >= 0");
    nrm += (double)v * (double)v;
  }
  free_graph(h);
  if (p.sweep_blocks > 0) {
    rc = build_sweep(h, p.sweep_blocks);
    if (rc) return rc;
  }
  h->prm = p;
  h->alpha = alpha;
  h->lam = relaxation;
  h->beta0 = p.beta0 < 0.0 ? 0.1 * std::sqrt(nrm) : p.beta0;
  h->tab.c = p.c_cdl;
  CK(cudaMemcpyAsync(h->w.p, hw.data(), h->n * sizeof(float), cudaMemcpyHostToDevice, s));
  if (h->btab_alpha != alpha || h->btab_beta0 != h->beta0) {
    // asynchronous: no allocation or host synchronisation in a served begin
    launch_beta_table(h->part.p + h->off_btab, kBetaTable, h->beta0, alpha, s);
    CK(cudaGetLastError());
    h->btab_alpha = alpha;
    h->btab_beta0 = h->beta0;
  }
  CK(h->log.alloc(std::max(1, p.log_capacity)));
  DevState& d = h->st_host;
  std::memset(&d, 0, sizeof(d));
  d.beta0 = h->beta0;
  d.alpha = alpha;
  d.lam = relaxation;
  d.eta = p.eta;
  d.W_all = h->W_all;
  d.reductions = p.reductions;
  d.max_trials = p.max_trials;
  d.norm = p.cimmino_norm;
  d.grad_normalize = p.grad_normalize ? 1 : 0;
  d.log_cap = p.log_capacity;
  d.f_empty = f_empty(h);
  CK(cudaMemcpyAsync(h->st.p, &d, sizeof(DevState), cudaMemcpyHostToDevice, s));
  h->iters_run = 0;
  h->device_ms = 0.0;
  h->it_pending = false;
  if (p.use_graphs) {
    const int64_t before = h->launches;
    const size_t t0 = h->timers_used;
    h->capturing = true;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(h);
    cudaError_t e = cudaStreamEndCapture(s, &h->graph);
    h->capturing = false;
    if (e != cudaSuccess) {
      h->graph = nullptr;
      h->timers_used = t0;
      return cuda_fail(h, e, "graph capture");
    }
    h->graph_nodes = (int)(h->launches - before);
    h->launches = before;
    if (h->timing) {
      // the event-record nodes of the capture, matched to the kernels' timers
      size_t n = 0;
      CK(cudaGraphGetNodes(h->graph, nullptr, &n));
      std::vector<cudaGraphNode_t> nodes(n);
      CK(cudaGraphGetNodes(h->graph, nodes.data(), &n));
      std::vector<std::pair<cudaEvent_t, cudaGraphNode_t>> rec;
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        CK(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        rec.emplace_back(ev, nd);
      }
      auto node_of = [&](cudaEvent_t ev) -> cudaGraphNode_t {
        for (auto& r : rec)
          if (r.first == ev) return r.second;
        return nullptr;
      };
      h->gtimers.clear();
      for (size_t i = t0; i < h->timers_used; ++i) {
        GraphTimer g{node_of(h->timers[i].a), node_of(h->timers[i].b), h->timers[i].cls};
        if (!g.a || !g.b) {
          h->timers_used = t0;
          free_graph(h);
          return fail(h, FREDOPT_ERR_CUDA, "timed graph capture: event node missing");
        }
        h->gtimers.push_back(g);
      }
      h->timers_used = t0;  // captured, not recorded: no times to collect
      h->graph_timed = true;
    }
    CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
  }
  CK(cudaStreamSynchronize(s));
  h->begun = true;
  return FREDOPT_OK;
}

int fredopt_iterate(fredopt_t h, int iters) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "call fredopt_begin first");
  if (iters < 0) return fail(h, FREDOPT_ERR_INVALID_ARG, "iters < 0");
  if (iters == 0) return FREDOPT_OK;
  DeviceGuard dg(h->device);
  if (h->it_pending) {
    float ms = 0.f;
    CK(cudaEventSynchronize(h->ev_it1));
    if (cudaEventElapsedTime(&ms, h->ev_it0, h->ev_it1) == cudaSuccess) h->device_ms += ms;
    h->it_pending = false;
  }
  CK(cudaEventRecord(h->ev_it0, h->stream));
  for (int i = 0; i < iters; ++i) {
    if (h->gexec && h->graph_timed == h->timing) {
      // a timed graph records each kernel's events into fresh timers; the
      // update affects this and later launches only
      for (const GraphTimer& g : h->gtimers) {
        Timer& t = next_timer(h, g.cls);
        CK(cudaGraphExecEventRecordNodeSetEvent(h->gexec, g.a, t.a));
        CK(cudaGraphExecEventRecordNodeSetEvent(h->gexec, g.b, t.b));
      }
      CK(cudaGraphLaunch(h->gexec, h->stream));
      h->launches += h->graph_nodes;
    } else {
      enqueue_iteration(h);
      CK(cudaGetLastError());
    }
  }
  CK(cudaEventRecord(h->ev_it1, h->stream));
  h->it_pending = true;
  h->iters_run += iters;
  return FREDOPT_OK;
}

int fredopt_end(fredopt_t h, float* w_out, float* dose_out, float* letd_out, fredopt_report* rep,
                uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "call fredopt_begin first");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  const Geometry& G = h->geo;
  if (h->it_pending) {
    float ms = 0.f;
    CK(cudaEventSynchronize(h->ev_it1));
    if (cudaEventElapsedTime(&ms, h->ev_it0, h->ev_it1) == cudaSuccess) h->device_ms += ms;
    h->it_pending = false;
  }
  // final double-float-accumulated product over every row
  CK(h->y64.ensure(std::max<int64_t>(1, h->V)));
  float* dptr = nullptr;
  float* lptr = nullptr;
  if (dose_out || letd_out) {
    if (dev_ptr(flags)) {
      dptr = dose_out;
      lptr = letd_out;
    } else {
      CK(h->fout_a.ensure(std::max<int64_t>(1, h->V)));
      CK(h->fout_b.ensure(std::max<int64_t>(1, h->V)));
      dptr = dose_out ? h->fout_a.p : nullptr;
      lptr = letd_out ? h->fout_b.p : nullptr;
    }
  }
  CK(cudaMemsetAsync(h->y64.p, 0, std::max<int64_t>(1, h->V) * sizeof(double2), s));
  if (dptr) CK(cudaMemsetAsync(dptr, 0, h->V * sizeof(float), s));
  if (lptr) CK(cudaMemsetAsync(lptr, 0, h->V * sizeof(float), s));
  FwdArgs fa = fwd_args(h, false);
  fa.x = h->w.p;
  fa.y64 = h->y64.p;
  fa.dose_out = dptr;
  fa.letd_out = lptr;
  run(h, 0, [&] { launch_forward(G, h->fmt, EPI_FINAL, false, fa, h->tab, s); });
  double* pf = h->part.p + h->off_fin;
  run(h, 5, [&] { launch_final_check(G, h->tab, h->y64.p, h->mask.p, h->mdd.p, h->mll.p, h->mdl.p, h->n_hot, pf, s); });
  CK(cudaGetLastError());
  std::vector<double> hp(8 * G.row_blocks);
  CK(cudaMemcpyAsync(hp.data(), pf, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  DevState d;
  CK(cudaMemcpyAsync(&d, h->st.p, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(copy_out(h, w_out, h->w.p, (size_t)h->n * sizeof(float), flags));
  if (!dev_ptr(flags)) {
    if (dose_out) CK(cudaMemcpyAsync(dose_out, h->fout_a.p, h->V * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (letd_out) CK(cudaMemcpyAsync(letd_out, h->fout_b.p, h->V * sizeof(float), cudaMemcpyDeviceToHost, s));
  }
  rc = check_sticky(h);
  collect_timers(h);
  if (rc) return rc;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->iters = h->iters_run;
    rep->s = d.s;
    rep->accepted = d.accepted_total;
    rep->n_rows = h->n_rows_reach;
    rep->unreachable_rows = h->n_unreach;
    double nv = 0.0, f = 0.0;
    for (int b = 0; b < G.row_blocks; ++b) {
      for (int q = 0; q < 6; ++q) rep->max_violation[q] = std::max(rep->max_violation[q], hp[8 * b + q]);
      nv += hp[8 * b + 6];
      f += hp[8 * b + 7];
    }
    rep->n_violated = (int64_t)nv;
    rep->objective = f;
    rep->beta0 = h->beta0;
    rep->device_ms = h->device_ms;
  }
  return FREDOPT_OK;
}

int fredopt_superiorize(fredopt_t h, const float* w0, int iters, double alpha, double relaxation,
                        const fredopt_params* params, float* w_out, float* dose_out,
                        float* letd_out, fredopt_report* rep, uint32_t flags) {
  int rc = fredopt_begin(h, w0, alpha, relaxation, params, flags);
  if (rc) return rc;
  rc = fredopt_iterate(h, iters);
  if (rc) return rc;
  return fredopt_end(h, w_out, dose_out, letd_out, rep, flags);
}

int fredopt_get_log(fredopt_t h, fredopt_log_entry* out, int max_entries) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "no solve begun");
  if (max_entries < 0 || (max_entries > 0 && !out)) return fail(h, FREDOPT_ERR_INVALID_ARG, "bad output");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  DevState d;
  CK(cudaMemcpy(&d, h->st.p, sizeof(DevState), cudaMemcpyDeviceToHost));
  const int cap = h->prm.log_capacity;
  if (cap <= 0) return 0;
  const int64_t k = d.k;
  const int64_t first = std::max<int64_t>(0, k - cap);
  const int cnt = (int)std::min<int64_t>(k - first, max_entries);
  std::vector<LogEntry> all(cap);
  CK(cudaMemcpy(all.data(), h->log.p, cap * sizeof(LogEntry), cudaMemcpyDeviceToHost));
  for (int i = 0; i < cnt; ++i) {
    const LogEntry& e = all[(first + i) % cap];
    out[i].k = e.k;
    out[i].s = e.s;
    out[i].accepted = e.accepted;
    out[i].n_violated = e.n_violated;
    out[i].beta = e.beta;
    out[i].f_start = e.f_start;
    out[i].f_end = e.f_end;
    out[i].gnorm = e.gnorm;
    out[i].max_violation = e.max_violation;
  }
  return cnt;
}

int fredopt_get_state(fredopt_t h, float* w, int64_t* k, int64_t* s, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "no solve begun");
  DeviceGuard dg(h->device);
  DevState d;
  CK(cudaMemcpyAsync(&d, h->st.p, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  if (w) CK(copy_out(h, w, h->w.p, (size_t)h->n * sizeof(float), flags));
  rc = check_sticky(h);
  if (rc) return rc;
  if (k) *k = d.k;
  if (s) *s = d.s;
  return FREDOPT_OK;
}

int fredopt_set_state(fredopt_t h, const float* w, int64_t k, int64_t s, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->begun) return fail(h, FREDOPT_ERR_NOT_LOADED, "call fredopt_begin first");
  if (!w || k < 0 || s < 0) return fail(h, FREDOPT_ERR_INVALID_ARG, "bad state");
  DeviceGuard dg(h->device);
  join_in(h);
  CK(cudaStreamSynchronize(h->stream));
  DevState d;
  CK(cudaMemcpy(&d, h->st.p, sizeof(DevState), cudaMemcpyDeviceToHost));
  d.k = k;
  d.s = s;
  d.done = 0u;
  CK(copy_in(h, h->w.p, w, (size_t)h->n * sizeof(float), flags));
  h->st_host = d;
  CK(cudaMemcpyAsync(h->st.p, &h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FREDOPT_OK;
}

int fredopt_forward(fredopt_t h, const float* w, float* dose_out, float* lw_out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!w) return fail(h, FREDOPT_ERR_INVALID_ARG, "w is null");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  join_in(h);
  rc = load_spot_vec(h, h->xbuf, w, flags);
  if (rc) return rc;
  CK(h->yall.ensure(std::max<int64_t>(1, h->V)));
  CK(cudaMemsetAsync(h->yall.p, 0, std::max<int64_t>(1, h->V) * sizeof(float2), s));
  FwdArgs fa = fwd_args(h, false);
  fa.x = h->xbuf.p;
  fa.y = h->yall.p;
  run(h, 0, [&] { launch_forward(h->geo, h->fmt, EPI_STORE, h->hint_fwd, fa, h->tab, s); });
  float *da = dose_out, *db = lw_out;
  if (!dev_ptr(flags)) {
    CK(h->fout_a.ensure(std::max<int64_t>(1, h->V)));
    CK(h->fout_b.ensure(std::max<int64_t>(1, h->V)));
    da = dose_out ? h->fout_a.p : nullptr;
    db = lw_out ? h->fout_b.p : nullptr;
  }
  launch_scatter_y(h->yall.p, h->perm ? h->voxel.p : nullptr, h->V, da, db, s);
  CK(cudaGetLastError());
  if (!dev_ptr(flags)) {
    if (dose_out) CK(cudaMemcpyAsync(dose_out, h->fout_a.p, h->V * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (lw_out) CK(cudaMemcpyAsync(lw_out, h->fout_b.p, h->V * sizeof(float), cudaMemcpyDeviceToHost, s));
  }
  rc = check_sticky(h);
  collect_timers(h);
  return rc;
}

int fredopt_backward(fredopt_t h, const float* a_D, const float* a_L, float* u_out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!u_out) return fail(h, FREDOPT_ERR_INVALID_ARG, "u_out is null");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  join_in(h);
  const float *pa = a_D, *pb = a_L;
  if (!dev_ptr(flags)) {
    CK(h->vin_a.ensure(std::max<int64_t>(1, h->V)));
    CK(h->vin_b.ensure(std::max<int64_t>(1, h->V)));
    if (a_D) CK(cudaMemcpyAsync(h->vin_a.p, a_D, h->V * sizeof(float), cudaMemcpyHostToDevice, s));
    if (a_L) CK(cudaMemcpyAsync(h->vin_b.p, a_L, h->V * sizeof(float), cudaMemcpyHostToDevice, s));
    pa = a_D ? h->vin_a.p : nullptr;
    pb = a_L ? h->vin_b.p : nullptr;
  }
  CK(h->ucoef.ensure(std::max<int64_t>(1, h->n_hot)));
  launch_scale_coef(h->n_hot, pa, pb, h->perm ? h->voxel.p : nullptr, h->fmt ? h->sD.p : nullptr,
                    h->fmt ? h->sL.p : nullptr, h->ucoef.p, s);
  BwdArgs ba = bwd_args(h, h->ucoef.p);
  run(h, 1, [&] { launch_backward(h->geo, h->fmt, h->hint_bwd, true, ba, s); });
  ColArgs ca = col_args(h);
  ca.out = h->gtmp.p;
  run(h, 3, [&] { launch_colfinish(h->geo, COL_OUT, ca, s); });
  CK(cudaGetLastError());
  CK(copy_out(h, u_out, h->gtmp.p, (size_t)h->n * sizeof(float), flags));
  rc = check_sticky(h);
  collect_timers(h);
  return rc;
}

int fredopt_feasibility_step(fredopt_t h, const float* x, double relaxation, double prio_scale,
                             int norm, float* w_out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!h->have_con) return fail(h, FREDOPT_ERR_NOT_LOADED, "no constraints set");
  if (!x || !w_out || !(relaxation > 0.0 && relaxation <= 2.0) || !(prio_scale > 0.0) ||
      (norm != FREDOPT_NORM_ALL && norm != FREDOPT_NORM_VIOLATED))
    return fail(h, FREDOPT_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  const Geometry& G = h->geo;
  join_in(h);
  rc = load_spot_vec(h, h->xbuf, x, flags);
  if (rc) return rc;
  FwdArgs fa = fwd_args(h, true);
  fa.x = h->xbuf.p;
  fa.y = h->yw.p;
  run(h, 0, [&] { launch_forward(G, h->fmt, EPI_STORE, h->hint_fwd, fa, h->tab, s); });
  ConArgs k2 = con_args(h);
  run(h, 2, [&] { launch_constraints(G, h->tab, k2, s); });
  if (h->tab.n_con > 0) {
    BwdArgs bb = bwd_args(h, h->gam.p);
    run(h, 1, [&] { launch_backward(G, h->fmt, h->hint_bwd, true, bb, s); });
  }
  ColArgs cc = col_args(h);
  cc.w = h->xbuf.p;
  cc.use_u = h->tab.n_con > 0 ? 1 : 0;
  cc.norm = norm;
  cc.lam = relaxation;
  cc.prio_scale = prio_scale;
  cc.in_solve = 0;
  cc.has_scale = norm != FREDOPT_NORM_VIOLATED ? 1 : 0;
  cc.scale = h->W_all > 0.0 ? relaxation * prio_scale / h->W_all : 0.0;
  run(h, 3, [&] { launch_colfinish(G, COL_PROJ, cc, s); });
  CK(cudaGetLastError());
  CK(copy_out(h, w_out, h->xbuf.p, (size_t)h->n * sizeof(float), flags));
  rc = check_sticky(h);
  collect_timers(h);
  return rc;
}

int fredopt_sweep_step(fredopt_t h, const float* x, double relaxation, double prio_scale, int norm,
                       int n_blocks, float* w_out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!x || !w_out) return fail(h, FREDOPT_ERR_INVALID_ARG, "null x or w_out");
  if (!(relaxation > 0.0 && relaxation <= 2.0)) return fail(h, FREDOPT_ERR_INVALID_ARG, "need 0 < relaxation <= 2");
  if (norm != FREDOPT_NORM_ALL && norm != FREDOPT_NORM_VIOLATED) return fail(h, FREDOPT_ERR_INVALID_ARG, "bad norm");
  if (n_blocks < 1 || n_blocks > FREDOPT_MAX_SWEEP_BLOCKS)
    return fail(h, FREDOPT_ERR_INVALID_ARG, "need 1 <= n_blocks <= FREDOPT_MAX_SWEEP_BLOCKS");
  if (h->begun && h->gexec && h->prm.sweep_blocks > 0 && h->sweep_m != n_blocks)
    return fail(h, FREDOPT_ERR_INVALID_ARG, "the begun solve sweeps another number of blocks");
  DeviceGuard dg(h->device);
  join_in(h);
  rc = build_sweep(h, n_blocks);
  if (rc) return rc;
  rc = load_spot_vec(h, h->xbuf, x, flags);
  if (rc) return rc;
  CK(h->gtmp.ensure(h->n_pad));
  enqueue_sweep(h, h->xbuf.p, 0, relaxation, prio_scale, norm, 0, h->gtmp.p);
  CK(cudaGetLastError());
  CK(copy_out(h, w_out, h->gtmp.p, (size_t)h->n * sizeof(float), flags));
  rc = check_sticky(h);
  collect_timers(h);
  return rc;
}

int fredopt_objective(fredopt_t h, const float* x, double* f_out, float* grad_out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!x) return fail(h, FREDOPT_ERR_INVALID_ARG, "x is null");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  const Geometry& G = h->geo;
  join_in(h);
  rc = load_spot_vec(h, h->xbuf, x, flags);
  if (rc) return rc;
  double* part_f = h->part.p + h->off_f;
  FwdArgs fa = fwd_args(h, true);
  fa.x = h->xbuf.p;
  fa.y = h->yw.p;
  fa.r_out = h->r.p;
  fa.part = part_f;
  run(h, 0, [&] { launch_forward(G, h->fmt, EPI_OBJ, h->hint_fwd, fa, h->tab, s); });
  BwdArgs ba = bwd_args(h, h->r.p);
  run(h, 1, [&] { launch_backward(G, h->fmt, h->hint_bwd, h->obj_dose, ba, s); });
  ColArgs ca = col_args(h);
  ca.out = h->gtmp.p;
  ca.part = h->part.p + h->off_g;
  run(h, 3, [&] { launch_colfinish(G, COL_GRAD, ca, s); });
  CK(cudaGetLastError());
  std::vector<double> hp(fa.n_warps);
  CK(cudaMemcpyAsync(hp.data(), part_f, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad_out) CK(copy_out(h, grad_out, h->gtmp.p, (size_t)h->n * sizeof(float), flags));
  rc = check_sticky(h);
  collect_timers(h);
  if (rc) return rc;
  if (f_out) {
    double f = f_empty(h);
    for (double v : hp) f += v;
    *f_out = f;
  }
  return FREDOPT_OK;
}

int fredopt_volume_stats(fredopt_t h, const float* w, uint32_t flags, int n_req, fredopt_volume_request* req) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (n_req < 0 || n_req > FREDOPT_VOLUME_MAX_REQUESTS || (n_req > 0 && !req))
    return fail(h, FREDOPT_ERR_INVALID_ARG, "need 0 <= n_req <= FREDOPT_VOLUME_MAX_REQUESTS and req");
  VolArgs va{};
  SelArgs sa{};
  std::vector<float> edges;
  std::vector<double> fracs;
  std::vector<int> sel_req;
  int n_bins = 0;
  for (int i = 0; i < n_req; ++i) {
    const fredopt_volume_request& r = req[i];
    if (r.quantity < FREDOPT_Q_DOSE || r.quantity > FREDOPT_Q_LETD)
      return fail(h, FREDOPT_ERR_INVALID_ARG, "quantity must be FREDOPT_Q_DOSE, _CDL or _LETD");
    if (r.struct_bit < 0 || r.struct_bit > 31) return fail(h, FREDOPT_ERR_INVALID_ARG, "struct_bit must be 0..31");
    if (r.n_bins < 0 || r.n_fracs < 0) return fail(h, FREDOPT_ERR_INVALID_ARG, "negative n_bins or n_fracs");
    if (r.n_bins > 0 && (!r.edges || !r.counts)) return fail(h, FREDOPT_ERR_INVALID_ARG, "edges or counts is null");
    if (r.n_fracs > 0 && (!r.fracs || !r.at_volume))
      return fail(h, FREDOPT_ERR_INVALID_ARG, "fracs or at_volume is null");
    if (n_bins + (int64_t)r.n_bins > FREDOPT_VOLUME_MAX_BINS)
      return fail(h, FREDOPT_ERR_INVALID_ARG, "more than FREDOPT_VOLUME_MAX_BINS bins in total");
    if ((int64_t)fracs.size() + r.n_fracs > FREDOPT_VOLUME_MAX_FRACS)
      return fail(h, FREDOPT_ERR_INVALID_ARG, "more than FREDOPT_VOLUME_MAX_FRACS fractions in total");
    for (int b = 0; b <= r.n_bins && r.n_bins > 0; ++b) {
      if (std::isnan(r.edges[b])) return fail(h, FREDOPT_ERR_INVALID_ARG, "NaN edge");
      if (b > 0 && r.edges[b] < r.edges[b - 1]) return fail(h, FREDOPT_ERR_INVALID_ARG, "edges decrease");
    }
    for (int q = 0; q < r.n_fracs; ++q)
      if (!(r.fracs[q] > 0.0 && r.fracs[q] <= 1.0)) return fail(h, FREDOPT_ERR_INVALID_ARG, "fraction outside (0, 1]");
    va.q[i] = r.quantity;
    va.bit[i] = r.struct_bit;
    va.nb[i] = r.n_bins;
    va.eoff[i] = (int32_t)edges.size();
    va.boff[i] = n_bins;
    if (r.n_bins > 0) edges.insert(edges.end(), r.edges, r.edges + r.n_bins + 1);
    n_bins += r.n_bins;
    for (int q = 0; q < r.n_fracs; ++q) {
      const int j = (int)fracs.size();
      sa.q[j] = r.quantity;
      sa.bit[j] = r.struct_bit;
      sel_req.push_back(i);
      fracs.push_back(r.fracs[q]);
    }
    va.any_bits |= 1u << r.struct_bit;
  }
  if (n_req == 0) return FREDOPT_OK;
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  join_in(h);
  rc = final_pass_y64(h, w, flags);
  if (rc) return rc;

  // scratch: edges | counts | n_vox | digit histograms | selection slots
  const int n_sel = (int)fracs.size();
  const size_t o_edges = 0;
  const size_t o_counts = o_edges + align256(std::max<size_t>(1, edges.size()) * sizeof(float));
  const size_t o_nvox = o_counts + align256(std::max(1, n_bins) * sizeof(unsigned long long));
  const size_t o_hist = o_nvox + align256(n_req * sizeof(unsigned long long));
  const size_t o_slot = o_hist + align256(std::max(1, n_sel) * 256 * sizeof(uint32_t));
  const size_t total = o_slot + align256(std::max(1, n_sel) * sizeof(SelSlot));
  CK(h->vol_buf.ensure(total));
  uint8_t* base = h->vol_buf.p;
  CK(cudaMemsetAsync(base + o_counts, 0, o_slot - o_counts, s));
  if (!edges.empty())
    CK(cudaMemcpyAsync(base + o_edges, edges.data(), edges.size() * sizeof(float), cudaMemcpyHostToDevice, s));

  va.y64 = h->y64.p;
  va.mask = h->mask.p;
  va.n_rows = h->n_hot;  // every structure voxel is a streamed row
  va.c = h->tab.c;
  va.n_req = n_req;
  va.n_edges = (int)edges.size();
  va.n_bins = n_bins;
  va.edges = reinterpret_cast<const float*>(base + o_edges);
  va.counts = reinterpret_cast<unsigned long long*>(base + o_counts);
  va.n_vox = reinterpret_cast<unsigned long long*>(base + o_nvox);
  run(h, 5, [&] { launch_vol_hist(h->geo, va, s); });
  CK(cudaGetLastError());
  std::vector<unsigned long long> nvox(n_req);
  CK(cudaMemcpyAsync(nvox.data(), va.n_vox, n_req * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));

  std::vector<SelSlot> slots(std::max(1, n_sel));
  if (n_sel > 0) {
    for (int j = 0; j < n_sel; ++j) {
      const int64_t n = (int64_t)nvox[sel_req[j]];
      slots[j].prefix = 0u;
      slots[j].pad = 0u;
      slots[j].k = n > 0 ? (uint64_t)at_volume_rank(fracs[j], n) : 0u;
    }
    sa.y64 = h->y64.p;
    sa.mask = h->mask.p;
    sa.n_rows = h->n_hot;
    sa.c = h->tab.c;
    sa.any_bits = va.any_bits;
    sa.n_sel = n_sel;
    sa.hist = reinterpret_cast<uint32_t*>(base + o_hist);
    sa.st = reinterpret_cast<SelSlot*>(base + o_slot);
    CK(cudaMemcpyAsync(sa.st, slots.data(), n_sel * sizeof(SelSlot), cudaMemcpyHostToDevice, s));
    run(h, 5, [&] { launch_vol_select(h->geo, sa, s); });
    h->launches += 7;  // launch_vol_select enqueues 8 kernels
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(slots.data(), sa.st, n_sel * sizeof(SelSlot), cudaMemcpyDeviceToHost, s));
  }
  std::vector<unsigned long long> counts(std::max(1, n_bins));
  if (n_bins > 0)
    CK(cudaMemcpyAsync(counts.data(), va.counts, n_bins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  rc = check_sticky(h);
  collect_timers(h);
  if (rc) return rc;
  int j = 0;
  for (int i = 0; i < n_req; ++i) {
    fredopt_volume_request& r = req[i];
    r.n_voxels = (int64_t)nvox[i];
    for (int b = 0; b < r.n_bins; ++b) r.counts[b] = (int64_t)counts[va.boff[i] + b];
    for (int q = 0; q < r.n_fracs; ++q, ++j)
      r.at_volume[q] = nvox[i] > 0 ? key_to_float(slots[j].prefix) : std::numeric_limits<float>::quiet_NaN();
  }
  return FREDOPT_OK;
}

int fredopt_quantity_map(fredopt_t h, const float* w, int quantity, float* out, uint32_t flags) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (!out) return fail(h, FREDOPT_ERR_INVALID_ARG, "out is null");
  if (quantity < FREDOPT_Q_DOSE || quantity > FREDOPT_Q_LETD)
    return fail(h, FREDOPT_ERR_INVALID_ARG, "quantity must be FREDOPT_Q_DOSE, _CDL or _LETD");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  join_in(h);
  rc = final_pass_y64(h, w, flags);
  if (rc) return rc;
  float* dst = out;
  if (!dev_ptr(flags)) {
    CK(h->fout_a.ensure(std::max<int64_t>(1, h->V)));
    dst = h->fout_a.p;
  }
  run(h, 5, [&] { launch_vol_map(h->geo, h->y64.p, h->perm ? h->voxel.p : nullptr, h->V, quantity, h->tab.c, dst, s); });
  CK(cudaGetLastError());
  if (!dev_ptr(flags) && h->V > 0)
    CK(cudaMemcpyAsync(out, dst, h->V * sizeof(float), cudaMemcpyDeviceToHost, s));
  rc = check_sticky(h);
  collect_timers(h);
  return rc;
}

int fredopt_get_sizes(fredopt_t h, int64_t* n_vox, int64_t* n_spots, int64_t* nnz, int64_t* n_rows,
                      int64_t* nnz_rows) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (n_vox) *n_vox = h->V;
  if (n_spots) *n_spots = h->n;
  if (nnz) *nnz = h->nnz;
  if (n_rows) *n_rows = h->n_hot;
  if (nnz_rows) *nnz_rows = h->nnz_hot;
  return FREDOPT_OK;
}

int fredopt_get_storage(fredopt_t h, int* col_index_bytes, int* row_index_bytes, int* val_bytes) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (col_index_bytes) *col_index_bytes = h->col16.p ? 2 : 4;
  if (row_index_bytes) *row_index_bytes = h->crow16.p ? 2 : 4;
  if (val_bytes) *val_bytes = value_bytes(h->fmt);
  return FREDOPT_OK;
}

int fredopt_get_rows(fredopt_t h, int64_t* voxel, uint32_t* mask) {
  int rc = need_loaded(h);
  if (rc) return rc;
  DeviceGuard dg(h->device);
  if (voxel) {
    if (h->perm) {
      CK(cudaMemcpy(voxel, h->voxel.p, h->n_hot * sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
      for (int64_t i = 0; i < h->n_hot; ++i) voxel[i] = i;
    }
  }
  if (mask && h->n_hot) CK(cudaMemcpy(mask, h->mask.p, h->n_hot * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return FREDOPT_OK;
}

int fredopt_get_csc(fredopt_t h, int64_t* col_ptr, int32_t* row, float* D_val, float* L_val) {
  int rc = need_loaded(h);
  if (rc) return rc;
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  if (col_ptr) CK(cudaMemcpyAsync(col_ptr, h->cp.p, (h->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (row && h->nnz_hot) CK(cudaMemcpyAsync(row, h->crow.p, h->nnz_hot * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if ((D_val || L_val) && h->nnz_hot) {
    DBuf<float> a, b;
    CK(a.alloc(h->nnz_hot));
    CK(b.alloc(h->nnz_hot));
    launch_dequant_csc(h->fmt, h->cp.p, h->n, h->crow.p, h->DTv.p, h->LTv.p, h->fmt ? h->sD.p : nullptr,
                       h->fmt ? h->sL.p : nullptr, a.p, b.p, s);
    CK(cudaGetLastError());
    if (D_val) CK(cudaMemcpyAsync(D_val, a.p, h->nnz_hot * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (L_val) CK(cudaMemcpyAsync(L_val, b.p, h->nnz_hot * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaStreamSynchronize(s));
  return FREDOPT_OK;
}

int fredopt_get_moments(fredopt_t h, double* dd, double* ll, double* dl) {
  int rc = need_loaded(h);
  if (rc) return rc;
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  if (h->n_hot == 0) return FREDOPT_OK;
  if (dd) CK(cudaMemcpy(dd, h->mdd.p, h->n_hot * sizeof(double), cudaMemcpyDeviceToHost));
  if (ll) CK(cudaMemcpy(ll, h->mll.p, h->n_hot * sizeof(double), cudaMemcpyDeviceToHost));
  if (dl) CK(cudaMemcpy(dl, h->mdl.p, h->n_hot * sizeof(double), cudaMemcpyDeviceToHost));
  return FREDOPT_OK;
}

int fredopt_set_timing(fredopt_t h, int enable) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  collect_timers(h);
  h->timing = enable != 0;
  for (int i = 0; i < FREDOPT_KCLASS_N; ++i) {
    h->kms[i] = 0.0;
    h->klaunch[i] = 0;
  }
  h->launches = 0;
  return FREDOPT_OK;
}

int fredopt_get_timing(fredopt_t h, double* ms, int64_t* launches) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  collect_timers(h);
  for (int i = 0; i < FREDOPT_KCLASS_N; ++i) {
    if (ms) ms[i] = h->kms[i];
    if (launches) launches[i] = h->klaunch[i];
  }
  return FREDOPT_OK;
}

int64_t fredopt_launch_count(fredopt_t h) { return h ? h->launches : -1; }

int fredopt_kernel_arch(int device, int* fwd_binary, int* bwd_binary, int* ptx_version) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return FREDOPT_ERR_CUDA;
  }
  const cudaError_t e = kernel_arch(fwd_binary, bwd_binary, ptx_version);
  cudaSetDevice(cur);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FREDOPT_ERR_CUDA;
  }
  return FREDOPT_OK;
}

int fredopt_check_wait(fredopt_t h, int arrive, int spins, float* elapsed_ms) {
  if (!h) return FREDOPT_ERR_INVALID_ARG;
  if (spins < 0) return fail(h, FREDOPT_ERR_INVALID_ARG, "spins must be >= 0");
  DeviceGuard dg(h->device);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(h, FREDOPT_ERR_CUDA, "event create");
  }
  cudaEventRecord(e0, h->stream);
  launch_wait_check(arrive, spins, h->st.p, h->stream);
  cudaError_t e = cudaGetLastError();
  cudaEventRecord(e1, h->stream);
  const int rc = e != cudaSuccess ? cuda_fail(h, e, "wait check launch") : check_sticky(h);
  if (elapsed_ms) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.0f;
    *elapsed_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int fredopt_get_tuning(fredopt_t h, int64_t* row_cost, int64_t* chunk_cost) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (row_cost) *row_cost = h->row_cost;
  if (chunk_cost) *chunk_cost = h->chunk_cost;
  return FREDOPT_OK;
}

int fredopt_autotune(fredopt_t h, int reps, int64_t* row_cost, int64_t* chunk_cost) {
  int rc = need_loaded(h);
  if (rc) return rc;
  if (reps < 1 || h->timing) return fail(h, FREDOPT_ERR_INVALID_ARG, "reps >= 1, timing off");
  DeviceGuard dg(h->device);
  cudaStream_t s = h->stream;
  const Geometry& G = h->geo;
  // inputs: w of the solve if one is begun, else ones; coefficients 1
  if (!h->begun) {
    std::vector<float> ones(h->n, 1.0f);
    CK(cudaMemcpyAsync(h->xbuf.p, ones.data(), h->n * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  const float* x = h->begun ? h->w.p : h->xbuf.p;
  launch_scale_coef(h->n_hot, nullptr, nullptr, nullptr, nullptr, nullptr, h->gam.p, s);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_ms = [&](auto&& launch) -> float {
    launch();  // warm-up
    float best = 1e30f;
    for (int i = 0; i < reps; ++i) {
      cudaEventRecord(e0, s);
      launch();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  FwdArgs fa = fwd_args(h, true);
  fa.x = x;
  fa.y = h->yw.p;
  int64_t best_row = h->row_cost;
  float best_f = 1e30f;
  for (int64_t c : {16, 32, 64, 128, 256, 512}) {
    if ((rc = set_fwd_schedule(h, c))) break;
    const float t = time_ms([&] { launch_forward(G, h->fmt, EPI_STORE, h->hint_fwd, fa, h->tab, s); });
    if (t < best_f) { best_f = t; best_row = c; }
  }
  BwdArgs ba = bwd_args(h, h->gam.p);
  int64_t best_chunk = h->chunk_cost;
  float best_b = 1e30f;
  for (int64_t c : {4, 16, 64, 256, 1024}) {
    if (rc || (rc = set_bwd_schedule(h, c))) break;
    const float t = time_ms([&] { launch_backward(G, h->fmt, h->hint_bwd, true, ba, s); });
    if (t < best_b) { best_b = t; best_chunk = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = set_fwd_schedule(h, best_row))) return rc;
  if ((rc = set_bwd_schedule(h, best_chunk))) return rc;
  rc = check_sticky(h);
  if (rc) return rc;
  if (row_cost) *row_cost = best_row;
  if (chunk_cost) *chunk_cost = best_chunk;
  return FREDOPT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct fredopt_batch {
  int device = 0;
  cudaStream_t root = nullptr;
  std::vector<fredopt_t> hs;
  std::vector<int> nodes;
  cudaGraph_t graph = nullptr;      // one iteration of every plan
  cudaGraphExec_t exec = nullptr;
  int depth = 1;                    // iterations of every plan in graph_k
  cudaGraph_t graph_k = nullptr;
  cudaGraphExec_t exec_k = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<cudaEvent_t> joins;
  double ms = 0.0;
  bool pending = false;
};

namespace {
void batch_free(fredopt_batch* b) {
  if (b->root) cudaStreamSynchronize(b->root);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->exec_k) cudaGraphExecDestroy(b->exec_k);
  if (b->graph_k) cudaGraphDestroy(b->graph_k);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->fork, b->done, b->t0, b->t1})
    if (e) cudaEventDestroy(e);
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
}
}  // namespace

extern "C" {

int fredopt_batch_create(fredopt_batch_t* out, const fredopt_t* handles, int n) {
  return fredopt_batch_create_depth(out, handles, n, 1);
}

int fredopt_batch_create_depth(fredopt_batch_t* out, const fredopt_t* handles, int n, int depth) {
  if (!out || !handles || n < 1 || depth < 1 || depth > FREDOPT_BATCH_MAX_DEPTH) return FREDOPT_ERR_INVALID_ARG;
  *out = nullptr;
  const int dev = handles[0] ? handles[0]->device : -1;
  for (int i = 0; i < n; ++i) {
    fredopt_t h = handles[i];
    if (!h || !h->loaded || !h->begun || h->device != dev || h->timing) return FREDOPT_ERR_NOT_LOADED;
    for (int j = 0; j < i; ++j)
      if (handles[j] == h || handles[j]->stream == h->stream) return FREDOPT_ERR_INVALID_ARG;
  }
  DeviceGuard dg(dev);
  fredopt_batch* b = new fredopt_batch();
  b->device = dev;
  b->hs.assign(handles, handles + n);
  auto bad = [&](cudaError_t e) {
    batch_free(b);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FREDOPT_ERR_OOM : FREDOPT_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
  for (cudaEvent_t* ev : {&b->fork, &b->done})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return bad(e);
  if ((e = cudaEventCreate(&b->t0)) != cudaSuccess || (e = cudaEventCreate(&b->t1)) != cudaSuccess) return bad(e);
  b->joins.resize(n, nullptr);
  for (int i = 0; i < n; ++i) {
    if ((e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming)) != cudaSuccess) return bad(e);
    if ((e = cudaStreamSynchronize(handles[i]->stream)) != cudaSuccess) return bad(e);
  }
  // `iters` iterations of every plan as parallel branches of one graph (each
  // branch runs its plan's iterations in order, exactly as alone)
  auto capture = [&](int iters, cudaGraph_t* g, cudaGraphExec_t* x) -> cudaError_t {
    cudaError_t ce = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ce;
    cudaEventRecord(b->fork, b->root);
    for (int i = 0; i < n; ++i) {
      fredopt_t h = handles[i];
      cudaStreamWaitEvent(h->stream, b->fork, 0);
      const int64_t before = h->launches;
      for (int k = 0; k < iters; ++k) enqueue_iteration(h);
      if (iters == 1) b->nodes.push_back((int)(h->launches - before));
      h->launches = before;
      cudaEventRecord(b->joins[i], h->stream);
      cudaStreamWaitEvent(b->root, b->joins[i], 0);
    }
    ce = cudaStreamEndCapture(b->root, g);
    if (ce != cudaSuccess) {
      *g = nullptr;
      return ce;
    }
    return cudaGraphInstantiate(x, *g, 0);
  };
  if ((e = capture(1, &b->graph, &b->exec)) != cudaSuccess) return bad(e);
  b->depth = depth;
  if (depth > 1 && (e = capture(depth, &b->graph_k, &b->exec_k)) != cudaSuccess) return bad(e);
  *out = b;
  return FREDOPT_OK;
}

int fredopt_batch_iterate(fredopt_batch_t b, int iters) {
  if (!b || iters < 0) return FREDOPT_ERR_INVALID_ARG;
  if (iters == 0) return FREDOPT_OK;
  DeviceGuard dg(b->device);
  if (b->pending) {
    float ms = 0.f;
    cudaEventSynchronize(b->t1);
    if (cudaEventElapsedTime(&ms, b->t0, b->t1) == cudaSuccess) b->ms += ms;
    b->pending = false;
  }
  for (fredopt_t h : b->hs) {  // order after any work the caller queued on the plans
    cudaEventRecord(h->ev_join, h->stream);
    cudaStreamWaitEvent(b->root, h->ev_join, 0);
  }
  cudaEventRecord(b->t0, b->root);
  // whole graphs of `depth` iterations, then single iterations
  const int nk = b->exec_k ? iters / b->depth : 0;
  for (int i = 0; i < nk; ++i)
    if (cudaGraphLaunch(b->exec_k, b->root) != cudaSuccess) {
      cudaGetLastError();
      return FREDOPT_ERR_CUDA;
    }
  for (int i = nk * b->depth; i < iters; ++i)
    if (cudaGraphLaunch(b->exec, b->root) != cudaSuccess) {
      cudaGetLastError();
      return FREDOPT_ERR_CUDA;
    }
  cudaEventRecord(b->t1, b->root);
  b->pending = true;
  cudaEventRecord(b->done, b->root);
  for (size_t i = 0; i < b->hs.size(); ++i) {
    fredopt_t h = b->hs[i];
    cudaStreamWaitEvent(h->stream, b->done, 0);  // later calls on the plan see the iterations
    h->iters_run += iters;
    h->launches += (int64_t)iters * b->nodes[i];
  }
  return FREDOPT_OK;
}

int fredopt_batch_sync(fredopt_batch_t b, double* device_ms) {
  if (!b) return FREDOPT_ERR_INVALID_ARG;
  DeviceGuard dg(b->device);
  if (cudaStreamSynchronize(b->root) != cudaSuccess) {
    cudaGetLastError();
    return FREDOPT_ERR_CUDA;
  }
  if (b->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->t0, b->t1) == cudaSuccess) b->ms += ms;
    b->pending = false;
  }
  if (device_ms) *device_ms = b->ms;
  for (fredopt_t h : b->hs) {
    int err = 0;
    cudaMemcpy(&err, &h->st.p->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return FREDOPT_ERR_TIMEOUT;
  }
  return FREDOPT_OK;
}

int fredopt_batch_destroy(fredopt_batch_t b) {
  if (!b) return FREDOPT_ERR_INVALID_ARG;
  DeviceGuard dg(b->device);
  batch_free(b);
  return FREDOPT_OK;
}

int fredopt_superiorize_batch(const fredopt_t* handles, int n, const float* const* w0, int iters, double alpha,
                              double relaxation, const fredopt_params* params, float* const* w_out,
                              float* const* dose_out, float* const* letd_out, fredopt_report* reps,
                              uint32_t flags) {
  if (!handles || !w0 || n < 1) return FREDOPT_ERR_INVALID_ARG;
  fredopt_params p;
  if (params) p = *params;
  else fredopt_default_params(&p);
  p.use_graphs = 0;  // the batch graph replaces the per-plan graphs
  for (int i = 0; i < n; ++i) {
    const int rc = fredopt_begin(handles[i], w0[i], alpha, relaxation, &p, flags);
    if (rc) return rc;
  }
  fredopt_batch_t b = nullptr;
  int rc = fredopt_batch_create_depth(&b, handles, n, std::max(1, std::min(iters, FREDOPT_BATCH_DEPTH)));
  if (rc) return rc;
  rc = fredopt_batch_iterate(b, iters);
  if (!rc) rc = fredopt_batch_sync(b, nullptr);
  fredopt_batch_destroy(b);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    rc = fredopt_end(handles[i], w_out ? w_out[i] : nullptr, dose_out ? dose_out[i] : nullptr,
                     letd_out ? letd_out[i] : nullptr, reps ? &reps[i] : nullptr, flags);
    if (rc) return rc;
  }
  return FREDOPT_OK;
}

}  // extern "C"

namespace fo {
cudaStream_t handle_stream(fredopt_t h) { return h ? h->stream : nullptr; }
int handle_device(fredopt_t h) { return h ? h->device : -1; }
}  // namespace fo

extern "C" {

}  // extern "C"
