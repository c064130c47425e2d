// Internal declarations shared by the kernels and the C ABI of libfredopt.
// Device data layout (all in HBM).  Device order of rows: streamed rows with
// nonzeros, streamed rows without, other rows with nonzeros, other rows
// without (each group ascending by voxel; see fredopt_api.cu):
//   CSR   rp int64[V+1], col int32[nnz] or col16 uint16[nnz] (n <= 65536 with x
//         staged in shared memory; the int32 copy is then freed after the CSC
//         build), Dv/Lv VT[nnz], sD/sL float[V] (16-bit only);
//         col/D/L zero padded so whole 32*16-byte blocks past the end stay in bounds
//   CSC   cp int64[n+1], row int32[nnz_hot] (index of a streamed row), DTv/LTv VT[nnz_hot];
//         for the transposed product also row16 uint16[nnz_hot] offsets from
//         per-128-element block bases hdr int32 (wide blocks in ovf)
//   rows  voxel int64[V] (device row -> voxel), mask uint32[n_hot],
//         FP64 moments |D_i|^2, |L_i|^2, <D_i,L_i> [n_hot]
//   state w/g float[n], yw/yg/r/gam float2[n_hot], chunk_sum float[n_chunks],
//         per-warp/per-block FP64 partials, DevState, log ring
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

struct fredopt_ctx;

namespace fo {

constexpr int kMaxCon = 32;
// elements of zero padding after the last nonzero of every index/value array
// (covers the block alignment and the prefetched unit of the streaming loop)
constexpr int64_t kPadElems = 1024;
constexpr int kMaxObj = 32;

// constraint kinds (same numbering as the public header)
enum Kind { DOSE_MIN = 0, DOSE_MAX = 1, CDL_MIN = 2, CDL_MAX = 3, LETD_MIN = 4, LETD_MAX = 5 };

struct ConEntry {
  uint32_t bit;
  int32_t kind;
  double bound;
  double prio;
};
struct ObjEntry {
  uint32_t bit;
  int32_t q;  // 0 dose, 1 cDL
  double target;
  double weight;
};
struct Tables {
  int32_t n_con;
  int32_t n_obj;
  double c;  // cDL constant
  ConEntry con[kMaxCon];
  ObjEntry obj[kMaxObj];
};

// device-resident scalars of a solve
struct DevState {
  double coef;        // perturbed point x = w + coef * g
  double beta0, alpha, lam, eta, W_all;
  double f_start, f_cur, gnorm, beta_acc;
  double f_empty;     // objective of streamed rows with no nonzeros (constant)
  long long k, s, accepted_total;
  int accepted;       // accepted steps in the current iteration
  int reductions, max_trials, norm, grad_normalize, log_cap;
  int err;            // bit 0: bulk-copy wait timed out; bit 1: index out of range (FO_CHECKED builds)
  unsigned int done;  // last-block counter of the column finish
  int pad;
  double sweep_nv, sweep_mx;  // block-iterative sweep: violated rows and largest violation
  unsigned int done_fin;      // last-block counter of the scalar finish
  int pad2;
};

struct LogEntry {
  long long k, s;
  int accepted, n_violated;
  double beta, f_start, f_end, gnorm, max_violation;
};

// epilogue modes of the forward product
enum FwdEpi { EPI_STORE = 0, EPI_OBJ = 1, EPI_BC = 2, EPI_FINAL = 3 };
// modes of the column finish
enum ColMode { COL_OUT = 0, COL_GRAD = 1, COL_PROJ = 2 };

struct FwdArgs {
  int64_t n_elems;        // allocated elements of the streamed arrays
  const int64_t* rp;
  const int32_t* col;     // column indices, or null when col16 is set
  const uint16_t* col16;  // 16-bit column indices (x staged in shared memory only)
  const void* Dv;
  const void* Lv;
  const float* sD;       // row scales (16-bit storage) or null
  const float* sL;
  const int64_t* warp_row;  // [2 * n_warps]: row range [r0, r1) of each tile (nonempty rows)
  unsigned int* sched;      // null: warp w streams tile w; else [2] counters of claimed tiles
  const float* x;
  int32_t n_x;           // number of spots
  int32_t n_x_pad;       // padded to a multiple of 4 (bulk-copy size)
  float2* y;             // (Dx, Lx) per row, FP32 (EPI_STORE/OBJ/BC)
  const uint32_t* mask;  // per streamed row
  int64_t n_hot;
  float2* r_out;         // EPI_OBJ: objective residual, scaled for the CSC
  const float2* r_in;    // EPI_BC: residual of EPI_OBJ
  double* part;          // per-tile partials, stride n_warps (the tile count): [f] or [B', C']
  int32_t n_warps;        // number of tiles in warp_row (the partials' stride)
  DevState* st;
  // EPI_FINAL
  double2* y64;
  const int64_t* voxel;  // device row -> voxel or null (identity)
  float* dose_out;
  float* letd_out;
};

struct BwdArgs {
  DevState* st;
  int64_t n_rows;         // streamed rows (range of the row indices)
  int64_t n_elems;        // allocated elements of the streamed arrays
  int32_t n_ovf;          // overflow slots of wide blocks
  const int32_t* row;
  const uint16_t* row16;  // based 16-bit row offsets, or null (then row)
  const int32_t* hdr;     // per 128-element block: base row, or -1 - overflow slot
  const int32_t* ovf;     // 128 int32 rows per overflow slot
  const void* Dv;
  const void* Lv;
  const int64_t* chunk_ptr;   // [n_chunks + 1]
  const int32_t* warp_chunk;  // [n_warps + 1]: chunk range of each tile
  unsigned int* sched;        // null: warp w streams tile w; else [2] counters of claimed tiles
  const float2* coef;         // per streamed row
  float* chunk_sum;
  int32_t n_warps;            // number of tiles
};

struct ColArgs {
  const int32_t* col_chunk;  // [n + 1]
  const float* chunk_sum;
  int32_t n;
  float* out;                // COL_OUT / COL_GRAD (g)
  float* w;                  // COL_PROJ: updated in place
  const float* g;            // COL_PROJ: gradient for the perturbed point
  double* part;              // per-block partials (COL_GRAD: ||g||^2)
  const double* k2part;      // COL_PROJ: constraint-evaluation partials
  int32_t k2_blocks;
  int32_t use_coef;          // COL_PROJ: 1 if x = w + coef*g
  double prio_scale;         // COL_PROJ outside a solve (feasibility step)
  int32_t norm;              // FREDOPT_NORM_*
  double lam;
  double W_all;
  int32_t in_solve;          // COL_PROJ: 1 = scale from DevState (eta^k) and advance k
  int32_t has_scale;         // COL_PROJ: 1 = the scale lam ps / W is `scale` (norm ALL, eta^k = 1)
  double scale;
  int32_t log_block;         // COL_PROJ in a solve with has_scale: 1 = one extra block closes the
                             // iteration (no block reads k), instead of the last block to finish
  int32_t use_u;             // 0: no transposed product (no constraints): u = 0
  DevState* st;
  LogEntry* log;
};

struct ConArgs {
  const float2* yw;     // (Dw, Lw)
  const float2* yg;     // (Dg, Lg) or null
  const uint32_t* mask;
  const double* dd;
  const double* ll;
  const double* dl;
  const float* sD;
  const float* sL;
  int64_t r0;           // rows [r0, n_hot) are evaluated (0 for the whole set)
  int64_t n_hot;
  // when set, the rows evaluated are rows[0 .. n_list) instead (the rows
  // with a structure bit, ascending); every other row's gam stays 0
  const int64_t* rows;
  int64_t n_list;
  float2* gam;
  double* part;         // per-block: [sum p violated, n violated, max violation, sum p reachable]
  int32_t use_coef;
  DevState* st;
};

// ---------------------------------------------------------------- launches
// (implemented in fredopt_kernels.cu; all asynchronous on `s`)

struct Geometry {
  int n_sms;
  int fwd_threads;      // 512
  int fwd_blocks;       // n_sms
  int fwd_warps;
  int bwd_threads;      // 256
  int bwd_blocks;
  int bwd_warps;
  int row_threads;      // 256
  int row_blocks;       // constraint kernel blocks
  int col_threads;      // 256
  int col_blocks;
  size_t smem_limit;    // bytes of opt-in shared memory per block
};

int init_kernels(Geometry* g, int device);  // sets function attributes once per device
// binary and PTX architecture versions (major * 10 + minor) of the loaded
// forward and transposed-product kernels on the current device
cudaError_t kernel_arch(int* fwd_binary, int* bwd_binary, int* ptx_version);

bool forward_uses_smem(const Geometry& g, int n_x_pad);
void launch_forward(const Geometry& g, int fmt, int epi, bool stream_hint, const FwdArgs& a,
                    const Tables& t, cudaStream_t s);
void launch_backward(const Geometry& g, int fmt, bool stream_hint, bool use_D, const BwdArgs& a,
                     cudaStream_t s);
void launch_colfinish(const Geometry& g, int mode, const ColArgs& a, cudaStream_t s);
// grid 0: g.row_blocks CTAs (the partials' stride); otherwise that many
void launch_constraints(const Geometry& g, const Tables& t, const ConArgs& a, cudaStream_t s, int grid = 0);
constexpr int kFinishBlocks = 64;  // CTAs of the scalar finish; stage holds 4 * kFinishBlocks doubles
// btab[s] = beta0 alpha^s for s < n_btab (filled at fredopt_begin)
constexpr long long kBetaTable = 1 << 16;
void launch_beta_table(double* out, long long n, double beta0, double alpha, cudaStream_t s);
void launch_finish(int step, const double* part_f, int nf, const double* part_bc, int nbc,
                   const double* part_g, int ng, DevState* st, double* stage, const double* btab,
                   long long n_btab, cudaStream_t s);
void launch_count_rows(const Geometry& g, const Tables& t, const uint32_t* mask, const double* dd,
                       const double* ll, const double* dl, int64_t n_hot, double* part,
                       cudaStream_t s);
void launch_scatter_y(const float2* y, const int64_t* voxel, int64_t n, float* a, float* b,
                      cudaStream_t s);
void launch_apply_step(int64_t n_hot, int n, float* w, const float* g, float2* yw, const float2* yg,
                       const DevState* st, cudaStream_t s);
void launch_row_objective(const Geometry& g, const Tables& t, const float2* yw, const uint32_t* mask,
                          const float* sD, const float* sL, int64_t n_hot, float2* r_out,
                          double* part, cudaStream_t s);
void launch_final_check(const Geometry& g, const Tables& t, const double2* y64, const uint32_t* mask,
                        const double* dd, const double* ll, const double* dl, int64_t n_hot,
                        double* part, cudaStream_t s);
void launch_begin_state(DevState* st, cudaStream_t s);

// setup (K5)
void launch_validate(const int64_t* rp, const int32_t* col, const float* D, const float* L,
                     int64_t n_rows, int32_t n_cols, int64_t nnz, int* err, cudaStream_t s);
void launch_gather_rows(const int64_t* rp_src, const int64_t* src_row, const int64_t* rp_dst,
                        int64_t n_rows, const int32_t* col_src, const float* D_src,
                        const float* L_src, int32_t* col_dst, float* D_dst, float* L_dst,
                        cudaStream_t s);
void launch_quantize(int fmt, const int64_t* rp, int64_t n_rows, const float* D, const float* L,
                     void* qD, void* qL, float* sD, float* sL, cudaStream_t s);
void launch_moments(int fmt, const int64_t* rp, int64_t n_rows, const void* Dv, const void* Lv,
                    const float* sD, const float* sL, double* dd, double* ll, double* dl,
                    cudaStream_t s);
// blocked stable counting transpose of rows [0, n_rows)
void launch_csc_count(const int64_t* rp, const int32_t* col, const int64_t* blk_row, int n_blk,
                      int32_t n_cols, int32_t* cnt, cudaStream_t s);
void launch_csc_offsets(int32_t* cnt, int n_blk, int32_t n_cols, const int64_t* cp, cudaStream_t s);
// stable CSR -> CSC scatter; a bulk-copy wait that gives up sets bit 0 of *err
// rec: null, or csc_fill_rec_bytes(...) bytes per output entry of scratch
// (n_out entries): the fill then stores one record per entry and splits them
void launch_csc_fill(const Geometry& g, int fmt, const int64_t* rp, const int32_t* col, const void* Dv,
                     const void* Lv, const int64_t* blk_row, int n_blk, int32_t n_cols, int32_t* cursor,
                     int32_t* row_out, void* DT, void* LT, int* err, void* rec, int64_t n_out, cudaStream_t s);
// bytes per entry of the fill's record scratch for this plan, 0 for none
size_t csc_fill_rec_bytes(const Geometry& g, int fmt, int32_t n_cols);
void launch_csc_colsum(const int32_t* cnt, int n_blk, int32_t n_cols, int64_t* tot, cudaStream_t s);
void launch_dequant_csc(int fmt, const int64_t* cp, int32_t n_cols, const int32_t* row, const void* DT,
                        const void* LT, const float* sD, const float* sL, float* Dout, float* Lout,
                        cudaStream_t s);
void launch_scale_coef(int64_t n, const float* aD, const float* aL, const int64_t* voxel,
                       const float* sD, const float* sL, float2* coef, cudaStream_t s);

// ---- block-iterative sweep (fredopt_sweep.cu)
struct SweepArgs {
  const int64_t* pos0;   // [n]: first CSC position of each column at or after the block's first row
  const int64_t* pos1;   // [n]: same for the next block
  const int32_t* row;    // CSC row indices (streamed rows)
  const void* Dv;        // CSC values
  const void* Lv;
  const float2* gam;     // per streamed row (scaled like the transposed product's coefficients)
  float* x;              // [n], updated in place
  int32_t n;
  const double* k2part;  // constraint partials of the block (4 slices of k2_blocks)
  int32_t k2_blocks;
  int32_t norm;
  double lam;
  double prio_scale;     // outside a solve
  int32_t in_solve;      // 1: scale eta^k from DevState and count the block's violations
  DevState* st;
};

void launch_sweep_start(int n, const float* w, const float* g, int use_coef, float* x, DevState* st,
                        cudaStream_t s);
void launch_sweep_pos(const int64_t* cp, const int32_t* row, int32_t n, const int64_t* bounds, int n_bounds,
                      int64_t* pos, cudaStream_t s);
void launch_sweep_update(const Geometry& g, int fmt, const SweepArgs& a, cudaStream_t s);
void launch_sweep_finish(const Geometry& g, int n, const float* x, float* out, int in_solve, DevState* st,
                         LogEntry* log, cudaStream_t s);
// Based 16-bit CSC row indices over n_blk blocks of 128 elements (pass 1:
// bases, offsets, wide blocks marked and counted in *n_wide; pass 2: overflow
// slots of the n_wide marked blocks, *slot zeroed before).
void launch_narrow_rows(const int32_t* row, int64_t n_blk, uint16_t* row16, int32_t* hdr, unsigned int* n_wide,
                        cudaStream_t s);
void launch_narrow_rows_wide(const int32_t* row, int64_t n_blk, int32_t* hdr, int32_t* ovf, unsigned int* slot,
                             unsigned int n_wide, cudaStream_t s);
// out[i] = in[i] for i < n (in[i] < 65536), n a multiple of 4.
void launch_narrow_idx(const int32_t* in, uint16_t* out, int64_t n, cudaStream_t s);
// One CTA in the bounded wait of the bulk copies (spins <= 0: their bound).
void launch_wait_check(int arrive, int spins, DevState* st, cudaStream_t s);

// ---- volume statistics (fredopt_volume.cu)
constexpr int kMaxVolReq = 64;  // requests per call
constexpr int kMaxSel = 64;     // (request, fraction) selections per call

// histograms: request i bins its structure's values with the packed edges
// [eoff[i], eoff[i] + nb[i]] into the packed counts [boff[i], boff[i] + nb[i])
struct VolArgs {
  const double2* y64;       // FP64 (Dw, Lw) per device row
  const uint32_t* mask;     // per device row
  int64_t n_rows;
  double c;                 // cDL constant
  uint32_t any_bits;        // union of the requested structure bits
  int n_req, n_edges, n_bins;
  int32_t q[kMaxVolReq], bit[kMaxVolReq], nb[kMaxVolReq], eoff[kMaxVolReq], boff[kMaxVolReq];
  const float* edges;
  unsigned long long* counts;  // [n_bins], zeroed by the caller
  unsigned long long* n_vox;   // [n_req], zeroed by the caller
};

struct SelSlot {
  uint32_t prefix;  // key bits chosen so far (the answer's key after the last pass)
  uint32_t pad;
  uint64_t k;       // rank (1 = largest) among the values matching the prefix; 0 = empty
};

struct SelArgs {
  const double2* y64;
  const uint32_t* mask;
  int64_t n_rows;
  double c;
  uint32_t any_bits;
  int n_sel;
  int32_t q[kMaxSel], bit[kMaxSel];
  uint32_t* hist;  // [n_sel][256], zeroed by the caller
  SelSlot* st;     // [n_sel]
};

size_t vol_hist_smem(const VolArgs& a);
void launch_vol_hist(const Geometry& g, const VolArgs& a, cudaStream_t s);
void launch_vol_select(const Geometry& g, const SelArgs& a, cudaStream_t s);  // 8 launches
void launch_vol_map(const Geometry& g, const double2* y64, const int64_t* voxel, int64_t n_rows, int q, double c,
                    float* out, cudaStream_t s);

// handle internals used by the serving loop (fredopt_server.cu)
cudaStream_t handle_stream(::fredopt_ctx* h);
int handle_device(::fredopt_ctx* h);

}  // namespace fo
