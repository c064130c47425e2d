// Seeded synthetic influence-matrix generator: homogeneous water phantom,
// axis-aligned proton pencil-beam fields, analytic depth dose and LET.
//
// This file produces INPUTS only (the dose-influence matrix D, Gy per unit
// spot weight, and the LET-weighted matrix L = LET_ij * D_ij, Gy*keV/um, in
// CSR with one shared sparsity pattern). It contains none of the
// optimisation method's arithmetic and is used by both the CUDA path and the
// FP64 oracle.  It stands in for Monte Carlo influence matrices (Sec. 2.2),
// which store the additive numerator and denominator of Eq. (1) per pencil
// beam; here the denominator is the dose itself.
//
// Physics (textbook, not from the paper):
//   * range-energy:  R = a * E^p, a = 0.0022 cm/MeV^p, p = 1.77 (Bragg-Kleeman)
//   * stopping power of the residual range r: S(r) = r^(1/p-1) / (p a^(1/p))
//   * fluence loss by nuclear interactions: (1 + b (R - z)) / (1 + b R),
//     b = 0.012 / cm
//   * range straggling: Gaussian in R with sigma_R = 0.012 * R^0.935 (cm)
//   * dose-averaged LET of one pencil beam at depth z:
//       int g Phi S^2 dR' / int g Phi S dR'  (MeV/cm -> keV/um: * 0.1),
//     capped at 15 keV/um
//   * lateral profile: exp(-(du^2+dv^2) / (2 sigma^2)), depth-independent
//   * truncation: keep (voxel, spot) if dd(z) * G >= trunc * max_z dd(z)
//   * noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
//     (seed, row, col); uniform multiplicative factors 1 + eps*(2u-1) on the
//     dose and on the LET; the sparsity pattern is noise-independent.
//
// Geometry: voxel (i, j, k) has centre ((i+.5)h, (j+.5)h, (k+.5)h) mm and
// row index (k*ny + j)*nx + i.  Beam angles are multiples of 90 degrees in
// the x-z plane: 0 -> +z, 90 -> +x, 180 -> -z, 270 -> -x.  Spot id =
// field*(layers*sy*sx) + layer*(sy*sx) + iy*sx + ix, so the columns of a row
// come out sorted when generated in (field, layer, iy, ix) order.
//
// Built as a plain host shared library (no intrinsics, portable to aarch64).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>

namespace {

constexpr double kA = 0.0022;   // cm / MeV^p
constexpr double kP = 1.77;
constexpr double kBeta = 0.012; // 1/cm
constexpr double kLetCap = 15.0; // keV/um
constexpr int kMaxFields = 8;

struct Table {
  double R_cm = 0;      // nominal range
  double dz_cm = 0;     // table step
  int n = 0;
  std::vector<double> dd;   // depth dose (arbitrary units)
  std::vector<double> let;  // keV/um
  double dd_max = 0;
  double z_end_cm = 0;      // dose is zero beyond
};

// integral of (x)^e over x in [lo, hi], lo, hi >= 0
inline double pow_integral(double lo, double hi, double e) {
  const double e1 = e + 1.0;
  return (std::pow(hi, e1) - std::pow(lo, e1)) / e1;
}

Table make_table(double R_cm, double dz_cm) {
  Table t;
  t.R_cm = R_cm;
  t.dz_cm = dz_cm;
  const double sR = 0.012 * std::pow(R_cm, 0.935);
  const double Rlo = std::max(R_cm - 5.0 * sR, 1e-6), Rhi = R_cm + 5.0 * sR;
  t.z_end_cm = Rhi;
  t.n = (int)std::ceil(Rhi / dz_cm) + 2;
  t.dd.assign(t.n, 0.0);
  t.let.assign(t.n, 0.0);
  const int M = 200;                      // straggling cells
  const double dR = (Rhi - Rlo) / M;
  const double q = 1.0 / kP - 1.0;        // exponent of S(r)
  const double inv_pa = 1.0 / (kP * std::pow(kA, 1.0 / kP));
  for (int iz = 0; iz < t.n; ++iz) {
    const double z = iz * dz_cm;
    double num = 0.0, den = 0.0;
    for (int c = 0; c < M; ++c) {
      const double a = Rlo + c * dR, b = a + dR;
      if (b <= z) continue;
      const double Rc = 0.5 * (a + b);
      const double g = std::exp(-0.5 * (Rc - R_cm) * (Rc - R_cm) / (sR * sR));
      const double phi = (1.0 + kBeta * std::max(Rc - z, 0.0)) / (1.0 + kBeta * Rc);
      const double lo = std::max(a, z) - z, hi = b - z;
      den += g * phi * inv_pa * pow_integral(lo, hi, q) / dR;
      num += g * phi * inv_pa * inv_pa * pow_integral(lo, hi, 2.0 * q) / dR;
    }
    t.dd[iz] = den;
    t.let[iz] = den > 0.0 ? std::min(0.1 * num / den, kLetCap) : 0.0;
  }
  t.dd_max = *std::max_element(t.dd.begin(), t.dd.end());
  return t;
}

inline void table_lookup(const Table& t, double z_cm, double* dd, double* let) {
  if (z_cm < 0.0 || z_cm >= t.z_end_cm) { *dd = 0.0; *let = 0.0; return; }
  const double f = z_cm / t.dz_cm;
  int i = (int)f;
  if (i >= t.n - 1) { *dd = 0.0; *let = 0.0; return; }
  const double u = f - i;
  *dd = t.dd[i] * (1.0 - u) + t.dd[i + 1] * u;
  *let = t.let[i] * (1.0 - u) + t.let[i + 1] * u;
}

// ---- Philox4x32-10 (published constants) ----
struct U4 { uint32_t v[4]; };
inline void mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}
inline U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(0xD2511F53u, ctr.v[0], &hi0, &lo0);
    mulhilo(0xCD9E8D57u, ctr.v[2], &hi1, &lo1);
    U4 n;
    n.v[0] = hi1 ^ ctr.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ ctr.v[3] ^ k1;
    n.v[3] = lo0;
    ctr = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return ctr;
}
inline double u01(uint32_t x) { return (x + 0.5) * (1.0 / 4294967296.0); }

}  // namespace

extern "C" {

// Parameters of one synthetic plan.  All lengths in mm.
struct phantom_params {
  int32_t nx, ny, nz;
  double h_mm;
  int32_t n_fields;
  double angle_deg[kMaxFields];
  double iso_mm[3];              // beam isocentre (lateral spot grid centre)
  int32_t spots_x, spots_y;      // lateral spot grid per field
  double spot_pitch_mm;
  int32_t n_layers;              // energy layers per field
  double range_first_mm[kMaxFields];  // nominal range of the shallowest layer (WET)
  double range_last_mm[kMaxFields];   // nominal range of the deepest layer (WET)
  double sigma_mm;               // lateral Gaussian sigma
  double trunc_rel;              // truncation relative to each spot's maximum
  double noise_rel;              // multiplicative noise amplitude (0 = clean)
  uint64_t seed;
  double shift_mm[3];            // patient setup shift (patient moves by +shift)
  double density_scale;          // water-equivalent depth = density_scale * depth
  double dose_at_iso;            // w = 1 gives this dose (Gy) at the isocentre
  double table_dz_mm;            // depth-table resolution
  int32_t n_threads;             // 0 = hardware concurrency
};

}  // extern "C"

namespace {

struct Field {
  int dir;   // 0:+z 1:+x 2:-z 3:-x
  std::vector<Table> layers;
};

struct Gen {
  const phantom_params& p;
  std::vector<Field> fields;
  double amp = 1.0;
  int64_t n_spots_field = 0;
  double r_cut_mm = 0;

  explicit Gen(const phantom_params& pp) : p(pp) {
    const double dz_cm = (p.table_dz_mm > 0 ? p.table_dz_mm : 0.1) * 0.1;
    for (int f = 0; f < p.n_fields; ++f) {
      Field fd;
      const long a = std::lround(p.angle_deg[f]) % 360;
      fd.dir = (int)(((a + 360) % 360) / 90);
      for (int l = 0; l < p.n_layers; ++l) {
        const double R_mm = p.n_layers == 1 ? p.range_first_mm[f]
            : p.range_first_mm[f] + (p.range_last_mm[f] - p.range_first_mm[f]) * l / (p.n_layers - 1);
        fd.layers.push_back(make_table(R_mm * 0.1, dz_cm));
      }
      fields.push_back(std::move(fd));
    }
    n_spots_field = (int64_t)p.n_layers * p.spots_x * p.spots_y;
    r_cut_mm = p.sigma_mm * std::sqrt(2.0 * std::log(1.0 / p.trunc_rel));
    // Analytic normalisation at the isocentre (no shift, nominal density).
    double s = 0.0;
    for (int f = 0; f < p.n_fields; ++f) {
      double depth = iso_depth_mm(f);
      double lat = 0.0;
      for (int iy = 0; iy < p.spots_y; ++iy)
        for (int ix = 0; ix < p.spots_x; ++ix) {
          const double du = spot_u(ix), dv = spot_v(iy);
          lat += std::exp(-(du * du + dv * dv) / (2.0 * p.sigma_mm * p.sigma_mm));
        }
      for (const Table& t : fields[f].layers) {
        double dd, let;
        table_lookup(t, depth * 0.1, &dd, &let);
        s += dd * lat;
      }
    }
    amp = s > 0.0 ? p.dose_at_iso / s : 1.0;
  }

  double spot_u(int ix) const { return (ix - 0.5 * (p.spots_x - 1)) * p.spot_pitch_mm; }
  double spot_v(int iy) const { return (iy - 0.5 * (p.spots_y - 1)) * p.spot_pitch_mm; }

  double iso_depth_mm(int f) const {
    const double X = p.nx * p.h_mm, Z = p.nz * p.h_mm;
    switch (fields[f].dir) {
      case 0: return p.iso_mm[2];
      case 1: return p.iso_mm[0];
      case 2: return Z - p.iso_mm[2];
      default: return X - p.iso_mm[0];
    }
  }

  // beam's-eye-view coordinates of a point (after the setup shift)
  void bev(int f, double x, double y, double z, double* u, double* v, double* depth) const {
    const double X = p.nx * p.h_mm, Z = p.nz * p.h_mm;
    x += p.shift_mm[0]; y += p.shift_mm[1]; z += p.shift_mm[2];
    *v = y - p.iso_mm[1];
    switch (fields[f].dir) {
      case 0: *u = x - p.iso_mm[0]; *depth = z; break;
      case 1: *u = -(z - p.iso_mm[2]); *depth = x; break;
      case 2: *u = -(x - p.iso_mm[0]); *depth = Z - z; break;
      default: *u = z - p.iso_mm[2]; *depth = X - x; break;
    }
    *depth *= p.density_scale;
  }

  // Visit the nonzeros of row r in column order.  emit(col, dose, let, key).
  template <class Emit>
  void row(int64_t r, Emit&& emit) const {
    const int64_t i = r % p.nx, j = (r / p.nx) % p.ny, k = r / ((int64_t)p.nx * p.ny);
    const double x = (i + 0.5) * p.h_mm, y = (j + 0.5) * p.h_mm, z = (k + 0.5) * p.h_mm;
    const double inv2s2 = 1.0 / (2.0 * p.sigma_mm * p.sigma_mm);
    for (int f = 0; f < p.n_fields; ++f) {
      double u, v, depth;
      bev(f, x, y, z, &u, &v, &depth);
      if (depth < 0.0) continue;
      const double cx = u / p.spot_pitch_mm + 0.5 * (p.spots_x - 1);
      const double cy = v / p.spot_pitch_mm + 0.5 * (p.spots_y - 1);
      const double rr = r_cut_mm / p.spot_pitch_mm;
      const int ix0 = std::max(0, (int)std::ceil(cx - rr)), ix1 = std::min(p.spots_x - 1, (int)std::floor(cx + rr));
      const int iy0 = std::max(0, (int)std::ceil(cy - rr)), iy1 = std::min(p.spots_y - 1, (int)std::floor(cy + rr));
      if (ix0 > ix1 || iy0 > iy1) continue;
      for (int l = 0; l < p.n_layers; ++l) {
        const Table& t = fields[f].layers[l];
        double dd, let;
        table_lookup(t, depth * 0.1, &dd, &let);
        if (dd <= 0.0) continue;
        const double thr = p.trunc_rel * t.dd_max;
        if (dd < thr) continue;
        for (int iy = iy0; iy <= iy1; ++iy) {
          const double dv = v - spot_v(iy);
          for (int ix = ix0; ix <= ix1; ++ix) {
            const double du = u - spot_u(ix);
            const double G = std::exp(-(du * du + dv * dv) * inv2s2);
            const double val = dd * G;
            if (val < thr) continue;
            const int64_t col = f * n_spots_field + (int64_t)l * p.spots_x * p.spots_y + (int64_t)iy * p.spots_x + ix;
            emit(col, amp * val, let);
          }
        }
      }
    }
  }
};

template <class F>
void parallel_rows(int64_t n_rows, int n_threads, F&& fn) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  n_threads = (int)std::min<int64_t>(n_threads, std::max<int64_t>(1, n_rows / 64));
  if (n_threads <= 1) { fn(0, n_rows); return; }
  std::vector<std::thread> th;
  // interleaved chunks for balance
  const int64_t chunk = 256;
  std::vector<int64_t> dummy;
  for (int t = 0; t < n_threads; ++t) {
    th.emplace_back([&, t]() {
      for (int64_t c0 = (int64_t)t * chunk; c0 < n_rows; c0 += (int64_t)n_threads * chunk)
        fn(c0, std::min(n_rows, c0 + chunk));
    });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

int64_t phantom_n_spots(const phantom_params* p) {
  return (int64_t)p->n_fields * p->n_layers * p->spots_x * p->spots_y;
}

int64_t phantom_n_voxels(const phantom_params* p) {
  return (int64_t)p->nx * p->ny * p->nz;
}

// Dose amplitude chosen by the analytic isocentre normalisation.
double phantom_amplitude(const phantom_params* p) {
  Gen g(*p);
  return g.amp;
}

// Depth-dose / LET table of one layer for inspection (n samples from z = 0).
int phantom_layer_table(const phantom_params* p, int field, int layer, int n, double* dd, double* let) {
  if (field < 0 || field >= p->n_fields || layer < 0 || layer >= p->n_layers) return -1;
  Gen g(*p);
  const Table& t = g.fields[field].layers[layer];
  for (int i = 0; i < n; ++i) {
    dd[i] = i < t.n ? t.dd[i] : 0.0;
    let[i] = i < t.n ? t.let[i] : 0.0;
  }
  return t.n;
}

// Pass 1: number of nonzeros per row.
int phantom_count(const phantom_params* p, int64_t* row_nnz) {
  if (p->n_fields < 1 || p->n_fields > kMaxFields) return -1;
  Gen g(*p);
  const int64_t V = phantom_n_voxels(p);
  parallel_rows(V, p->n_threads, [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      int64_t c = 0;
      g.row(r, [&](int64_t, double, double) { ++c; });
      row_nnz[r] = c;
    }
  });
  return 0;
}

// Pass 2: fill CSR values at the offsets given by row_ptr (from pass 1).
int phantom_fill(const phantom_params* p, const int64_t* row_ptr, int32_t* col, float* D, float* L) {
  if (p->n_fields < 1 || p->n_fields > kMaxFields) return -1;
  Gen g(*p);
  const int64_t V = phantom_n_voxels(p);
  const uint32_t k0 = (uint32_t)p->seed, k1 = (uint32_t)(p->seed >> 32);
  const double eps = p->noise_rel;
  parallel_rows(V, p->n_threads, [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      int64_t o = row_ptr[r];
      g.row(r, [&](int64_t c, double d, double let) {
        if (eps != 0.0) {
          U4 ctr{{(uint32_t)r, (uint32_t)(r >> 32), (uint32_t)c, 0x4C455444u}};
          const U4 o4 = philox4x32_10(ctr, k0, k1);
          d *= 1.0 + eps * (2.0 * u01(o4.v[0]) - 1.0);
          let *= 1.0 + eps * (2.0 * u01(o4.v[1]) - 1.0);
        }
        col[o] = (int32_t)c;
        D[o] = (float)d;
        L[o] = (float)(let * d);
        ++o;
      });
    }
  });
  return 0;
}

// Philox4x32-10 on one counter, exposed for the published known-answer test.
void phantom_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  U4 c{{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 o = philox4x32_10(c, key[0], key[1]);
  std::memcpy(out, o.v, sizeof(o.v));
}

}  // extern "C"
