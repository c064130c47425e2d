// Transposed product u = D^T a_D + L^T a_L over caller-owned device arrays
// without any device allocation.
//
// Some callers of this library cannot allocate device memory at the point
// where they need the product: a host application that hands every byte of
// the GPU to its own memory pool (so a stray cudaMalloc would fail or
// fragment the pool), or a latency-critical loop in which cudaMalloc and
// cudaFree are avoided because they can synchronise the device and stall
// work already queued.  This entry point needs no handle and no allocation:
// its scratch (per-column chunk offsets and per-chunk partial sums) is one
// fixed file-scope device array, held by every GPU that loads the library
// until the process exits.
//
// The work is split like the library's transposed product: each column is cut
// into chunks of kNaChunk nonzeros, every chunk is summed by one warp in a
// fixed order, and the chunk sums of a column are added in chunk order, so
// the result is deterministic.
#include "fredopt.h"

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace {

constexpr int kNaChunk = 4096;          // nonzeros per chunk
constexpr int kNaMaxCols = 65536;       // largest n_cols accepted
constexpr int kNaMaxChunks = 1 << 20;   // largest number of chunks accepted
constexpr size_t kNaOffBytes = ((size_t)(kNaMaxCols + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
constexpr size_t kNaScratchBytes = kNaOffBytes + (size_t)kNaMaxChunks * sizeof(float);

// The scratch: chunk offsets (int32[n_cols + 1]) then chunk sums
// (float[kNaMaxChunks]).  4.25 MiB.  Every call rewrites the parts it reads,
// so nothing has to start at zero.
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
void* g_na_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (cudaGetSymbolAddress with that device current) and kept for the
// life of the process.  A cudaDeviceReset reloads the module, so the kept
// address is no longer valid after one.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

__device__ __forceinline__ int64_t clamp_ptr(int64_t v, int64_t nnz) {
  return v < 0 ? 0 : (v > nnz ? nnz : v);
}

// Exclusive scan of the per-column chunk counts (one block).
__global__ void __launch_bounds__(1024) k_na_offsets(const int64_t* __restrict__ col_ptr, int32_t n_cols,
                                                     int64_t nnz, int32_t* __restrict__ off) {
  __shared__ int32_t sh[1024];
  int32_t carry = 0;
  for (int32_t base = 0; base < n_cols; base += 1024) {
    const int32_t j = base + threadIdx.x;
    int32_t c = 0;
    if (j < n_cols) {
      const int64_t s = clamp_ptr(col_ptr[j], nnz);
      int64_t e = clamp_ptr(col_ptr[j + 1], nnz);
      if (e < s) e = s;
      c = (int32_t)((e - s + kNaChunk - 1) / kNaChunk);
    }
    sh[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
      const int32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (j < n_cols) off[j] = carry + sh[threadIdx.x] - c;
    carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n_cols] = carry;
}

// One warp per chunk: sum of D_ij a_D[i] + L_ij a_L[i] over the chunk.
__global__ void __launch_bounds__(256) k_na_chunks(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row,
                                                   const float* __restrict__ Dv, const float* __restrict__ Lv,
                                                   const float* __restrict__ aD, const float* __restrict__ aL,
                                                   int64_t n_rows, int32_t n_cols, int64_t nnz,
                                                   const int32_t* __restrict__ off, float* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t total = off[n_cols];
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += nw) {
    int32_t lo = 0, hi = n_cols;  // last column j with off[j] <= g
    while (hi - lo > 1) {
      const int32_t m = (lo + hi) >> 1;
      if (off[m] <= g) lo = m;
      else hi = m;
    }
    const int32_t j = lo;
    const int64_t s0 = clamp_ptr(col_ptr[j], nnz);
    int64_t e0 = clamp_ptr(col_ptr[j + 1], nnz);
    if (e0 < s0) e0 = s0;
    const int64_t s = s0 + (int64_t)(g - off[j]) * kNaChunk;
    const int64_t e = s + kNaChunk < e0 ? s + kNaChunk : e0;
    float acc = 0.0f;
    for (int64_t p = s + lane; p < e; p += 32) {
      const int32_t r = row[p];
      if (r < 0 || r >= n_rows) continue;  // never read outside the coefficient arrays
      if (aD) acc = fmaf(Dv[p], aD[r], acc);
      if (aL) acc = fmaf(Lv[p], aL[r], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[g] = acc;
  }
}

// u_j = sum of the chunk sums of column j, in chunk order.
__global__ void k_na_columns(const int32_t* __restrict__ off, const float* __restrict__ part, int32_t n_cols,
                             float* __restrict__ u) {
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_cols; j += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int32_t g = off[j]; g < off[j + 1]; ++g) s += part[g];
    u[j] = s;
  }
}

}  // namespace

extern "C" int fredopt_backward_noalloc(int64_t n_rows, int32_t n_cols, int64_t nnz, const int64_t* col_ptr,
                                        const int32_t* row, const float* D_val, const float* L_val,
                                        const float* a_D, const float* a_L, float* u_out, void* cuda_stream) {
  if (n_rows < 0 || n_cols < 1 || nnz < 0) return FREDOPT_ERR_SHAPE;
  if (n_cols > kNaMaxCols || nnz / kNaChunk + n_cols > kNaMaxChunks) return FREDOPT_ERR_SHAPE;
  if (!col_ptr || !u_out || (nnz > 0 && (!row || !D_val || !L_val))) return FREDOPT_ERR_INVALID_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return FREDOPT_ERR_CUDA;
  }
  int32_t* off = reinterpret_cast<int32_t*>(base);
  float* part = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(base) + kNaOffBytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // grid of the chunk kernel: 8 CTAs per SM (152 SMs on GB300 if the query fails)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  k_na_offsets<<<1, 1024, 0, s>>>(col_ptr, n_cols, nnz, off);
  k_na_chunks<<<sms * 8, 256, 0, s>>>(col_ptr, row, D_val, L_val, a_D, a_L, n_rows, n_cols, nnz, off, part);
  k_na_columns<<<(n_cols + 255) / 256, 256, 0, s>>>(off, part, n_cols, u_out);
  if (cudaGetLastError() != cudaSuccess) return FREDOPT_ERR_CUDA;
  return FREDOPT_OK;
}
