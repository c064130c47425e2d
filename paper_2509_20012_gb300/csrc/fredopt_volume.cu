// Volume statistics of a plan (Sec. 2.4.1): per-structure histograms of
// dose, LETd and cDL (DVH, LVH, cDLVH) and the value received by a fraction
// of a structure's volume (cDL30, D98), from the FP64 final pass y64.
//
// Both kernels stream the device rows once per launch: mask (4 B) and y64
// (16 B) per row, reading y64 only for rows inside some requested structure.
// Counts are integers added with atomics, so every result is exact and
// independent of the launch shape.  The value at volume is an exact radix
// selection over the 32-bit keys of the FP32 values: four passes of eight
// bits, each a digit histogram of the values that still match the chosen
// prefix, followed by a one-block pick of the digit that holds the k-th
// largest value.
#include "fredopt_internal.cuh"

#include <algorithm>

namespace fo {

namespace {

// Voxel value of quantity q from the FP64 pair (Dw, Lw), rounded once to FP32
// exactly as the final pass rounds its dose and LETd outputs.
__device__ __forceinline__ float vol_value(int q, double2 y, double c) {
  if (q == 0) return (float)y.x;
  if (q == 1) return (float)(c * y.y);
  return y.x > 0.0 ? (float)(y.y / y.x) : 0.0f;
}

// Order-preserving map of a float to an unsigned key (larger float, larger key).
__device__ __forceinline__ uint32_t vol_key(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(256) k_vol_hist(VolArgs a) {
  extern __shared__ uint32_t vsh[];
  float* se = reinterpret_cast<float*>(vsh);            // packed edges
  uint32_t* sc = vsh + a.n_edges;                       // packed bin counts
  uint32_t* sn = sc + a.n_bins;                         // voxels per request
  for (int j = threadIdx.x; j < a.n_edges; j += blockDim.x) se[j] = a.edges[j];
  for (int j = threadIdx.x; j < a.n_bins + a.n_req; j += blockDim.x) sc[j] = 0u;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n_rows; r += stride) {
    const uint32_t m = a.mask[r];
    if (!(m & a.any_bits)) continue;
    const double2 y = a.y64[r];
    for (int i = 0; i < a.n_req; ++i) {
      if (!((m >> a.bit[i]) & 1u)) continue;
      atomicAdd(&sn[i], 1u);
      const int nb = a.nb[i];
      if (nb == 0) continue;
      const float v = vol_value(a.q[i], y, a.c);
      const float* e = se + a.eoff[i];
      if (!(v >= e[0]) || !(v < e[nb])) continue;  // outside the binned range
      int lo = 0, hi = nb;                          // largest b < nb with e[b] <= v
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= v) lo = mid;
        else hi = mid;
      }
      atomicAdd(&sc[a.boff[i] + lo], 1u);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < a.n_bins; j += blockDim.x)
    if (sc[j]) atomicAdd(&a.counts[j], (unsigned long long)sc[j]);
  for (int j = threadIdx.x; j < a.n_req; j += blockDim.x)
    if (sn[j]) atomicAdd(&a.n_vox[j], (unsigned long long)sn[j]);
}

// Digit histogram of selection slot j over the values whose key matches the
// slot's prefix above bit `shift + 8`.
__global__ void __launch_bounds__(256) k_vol_digits(SelArgs a, int shift) {
  extern __shared__ uint32_t dsh[];  // [n_sel][256]
  for (int j = threadIdx.x; j < a.n_sel * 256; j += blockDim.x) dsh[j] = 0u;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n_rows; r += stride) {
    const uint32_t m = a.mask[r];
    if (!(m & a.any_bits)) continue;
    const double2 y = a.y64[r];
    for (int j = 0; j < a.n_sel; ++j) {
      if (!((m >> a.bit[j]) & 1u)) continue;
      const uint32_t key = vol_key(vol_value(a.q[j], y, a.c));
      if (shift < 24 && (key >> (shift + 8)) != (a.st[j].prefix >> (shift + 8))) continue;
      atomicAdd(&dsh[j * 256 + ((key >> shift) & 255u)], 1u);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < a.n_sel * 256; j += blockDim.x)
    if (dsh[j]) atomicAdd(&a.hist[j], dsh[j]);
}

// One thread per slot: the digit whose bucket holds the k-th largest of the
// matching values; k becomes the rank inside that bucket.  Clears the
// slot's histogram for the next pass.
__global__ void k_vol_pick(SelArgs a, int shift) {
  const int j = threadIdx.x;
  if (j >= a.n_sel) return;
  uint32_t* h = a.hist + j * 256;
  SelSlot& s = a.st[j];
  if (s.k > 0) {
    uint64_t cum = 0;
    for (int d = 255; d >= 0; --d) {
      if (cum + h[d] >= s.k) {
        s.prefix |= (uint32_t)d << shift;
        s.k -= cum;
        break;
      }
      cum += h[d];
    }
  }
  for (int d = 0; d < 256; ++d) h[d] = 0u;
}

__global__ void __launch_bounds__(256) k_vol_map(const double2* y64, const int64_t* voxel, int64_t n_rows, int q,
                                                 double c, float* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += stride)
    out[voxel ? voxel[r] : r] = vol_value(q, y64[r], c);
}

unsigned vol_grid(const Geometry& g, int64_t n_rows) {
  const int64_t want = (n_rows + 255) / 256;
  const int64_t cap = (int64_t)g.n_sms * 4;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

}  // namespace

size_t vol_hist_smem(const VolArgs& a) {
  return (size_t)(a.n_edges + a.n_bins + a.n_req) * sizeof(uint32_t);
}

void launch_vol_hist(const Geometry& g, const VolArgs& a, cudaStream_t s) {
  const size_t smem = vol_hist_smem(a);
  cudaFuncSetAttribute(k_vol_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_vol_hist<<<vol_grid(g, a.n_rows), 256, smem, s>>>(a);
}

void launch_vol_select(const Geometry& g, const SelArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)a.n_sel * 256 * sizeof(uint32_t);
  cudaFuncSetAttribute(k_vol_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int shift = 24; shift >= 0; shift -= 8) {
    k_vol_digits<<<vol_grid(g, a.n_rows), 256, smem, s>>>(a, shift);
    k_vol_pick<<<1, kMaxSel, 0, s>>>(a, shift);
  }
}

void launch_vol_map(const Geometry& g, const double2* y64, const int64_t* voxel, int64_t n_rows, int q, double c,
                    float* out, cudaStream_t s) {
  if (n_rows == 0) return;
  k_vol_map<<<vol_grid(g, n_rows), 256, 0, s>>>(y64, voxel, n_rows, q, c, out);
}

}  // namespace fo
