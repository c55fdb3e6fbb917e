// Setup kernels: value gathers, box-basis evaluation of P (Section 4), the unisolvence
// check, the inter-level injection P~ (Section 4) and the Galerkin products
// A_{l+1} = P^T A_l P (Sections 1 and 4).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace r3mg {

constexpr int kMaxP = 8;   // p' <= 8 (GLL table size)

struct GLLTable { double z[kMaxP + 1]; int pp; };

// 1-D Lagrange values at t on the GLL nodes z[0..pp].
__device__ __forceinline__ void lagrange_vals(const GLLTable& g, double t, double* L) {
  for (int a = 0; a <= g.pp; ++a) {
    double v = 1.0;
    for (int k = 0; k <= g.pp; ++k)
      if (k != a) v *= (t - g.z[k]) / (g.z[a] - g.z[k]);
    L[a] = v;
  }
}

// phi_q(x) for the box [lo, hi]: product of 1-D Lagrange values, q lexicographic, x fastest.
__device__ __forceinline__ double box_phi(const GLLTable& g, int dim, const double* x, const double* lo,
                                          const double* hi, int q) {
  if (g.pp == 0) return 1.0;
  double v = 1.0;
  const int nb1 = g.pp + 1;
  for (int a = 0; a < dim; ++a) {
    const double t = (x[a] - lo[a]) / (hi[a] - lo[a]);
    const int qa = q % nb1;
    q /= nb1;
    double w = 1.0;
    for (int k = 0; k <= g.pp; ++k)
      if (k != qa) w *= (t - g.z[k]) / (g.z[qa] - g.z[k]);
    v *= w;
  }
  return v;
}

__global__ void k_gather_vals(const int64_t* __restrict__ src, const double* __restrict__ csr, double* out,
                              int64_t m) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = src[k];
    out[k] = s >= 0 ? csr[s] : 0.0;
  }
}

// dinv[i] = 1 / A_ii on the fine level; flags a non-positive or non-finite diagonal.
__global__ void k_dinv_fine(const int64_t* __restrict__ diag_src, const double* __restrict__ csr, double* dinv,
                            int64_t n, int* status) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double a = csr[diag_src[k]];
    if (!(a > 0.0) || !isfinite(a)) atomicExch(status, 1);
    dinv[k] = 1.0 / a;
  }
}

// Coarse diagonal: row (B,q) has its diagonal in the slot s with nbr[s] == B, column s*b+q.
__global__ void k_dinv_coarse(const int64_t* __restrict__ nbr_ptr, const int64_t* __restrict__ nbr,
                              const int64_t* __restrict__ row_ptr, const double* __restrict__ vals, double* dinv,
                              int64_t nbox, int b, int* status) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nbox * b; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t B = r / b;
    const int q = (int)(r - B * b);
    int64_t lo = nbr_ptr[B], hi = nbr_ptr[B + 1] - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (nbr[mid] < B) lo = mid + 1; else hi = mid;
    }
    const int64_t s = lo - nbr_ptr[B];
    const double a = vals[row_ptr[r] + s * b + q];
    if (!(a > 0.0) || !isfinite(a)) atomicExch(status, 1);
    dinv[r] = 1.0 / a;
  }
}

// P_0 values: row k (tree order) holds phi_{box(k),q}(x_k), q = 0..b-1.
__global__ void k_p0_eval(const double* __restrict__ coords_tree, const int32_t* __restrict__ box_of_tree,
                          const double* __restrict__ lo, const double* __restrict__ hi, GLLTable g, int dim, int b,
                          double* P0, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * b; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / b;
    const int q = (int)(t - k * b);
    const int64_t B = box_of_tree[k];
    P0[t] = box_phi(g, dim, coords_tree + k * dim, lo + B * dim, hi + B * dim, q);
  }
}

// Unisolvence of level-1 boxes (Section 4, Remark on (m, M)): the Gram matrix V^T V of the
// owned-point evaluation matrix V must have a Cholesky factorisation with every pivot above
// 1e-12 times its largest diagonal entry.  One CTA per box, b <= 64.
__global__ void k_unisolvent(const double* __restrict__ P0, const int64_t* __restrict__ box_row, int64_t nbox,
                             int b, int* status) {
  extern __shared__ double Gm[];
  __shared__ double s_tol;
  __shared__ int s_bad;
  for (int64_t B = blockIdx.x; B < nbox; B += gridDim.x) {
    const int64_t r0 = box_row[B], r1 = box_row[B + 1];
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
      const int i = t / b, j = t % b;
      double s = 0.0;
      for (int64_t k = r0; k < r1; ++k) s += P0[k * b + i] * P0[k * b + j];
      Gm[t] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int i = 0; i < b; ++i) mx = fmax(mx, Gm[i * b + i]);
      s_tol = 1e-12 * mx;
      s_bad = 0;
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {       // in-place lower Cholesky, column j
      if (threadIdx.x == 0) {
        double s = Gm[j * b + j];
        for (int k = 0; k < j; ++k) s -= Gm[j * b + k] * Gm[j * b + k];
        if (!(s > s_tol)) s_bad = 1;
        Gm[j * b + j] = sqrt(fmax(s, 1e-300));
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) {
        double s = Gm[i * b + j];
        for (int k = 0; k < j; ++k) s -= Gm[i * b + k] * Gm[j * b + k];
        Gm[i * b + j] = s / Gm[j * b + j];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && s_bad) atomicExch(status, 1);
    __syncthreads();
  }
}

// P~_l block of child c: Pt[c][q'][q] = phi_{parent(c), q}(xi_{c,q'}), xi = child's GLL nodes.
__global__ void k_ptilde_eval(const double* __restrict__ lo_c, const double* __restrict__ hi_c,
                              const double* __restrict__ lo_p, const double* __restrict__ hi_p, GLLTable g, int dim,
                              int b, int fan, double* Pt, int64_t nchild) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nchild * b * b;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / (b * b);
    const int rem = (int)(t - c * b * b);
    const int qp = rem / b, q = rem % b;
    const int64_t B = c / fan;
    double xi[3];
    int r = qp;
    const int nb1 = g.pp + 1;
    for (int a = 0; a < dim; ++a) {
      const double l = lo_c[c * dim + a], h = hi_c[c * dim + a];
      xi[a] = (g.pp == 0) ? 0.5 * (l + h) : l + g.z[r % nb1] * (h - l);
      r /= nb1;
    }
    Pt[t] = box_phi(g, dim, xi, lo_p + B * dim, hi_p + B * dim, q);
  }
}

// Galerkin product for the fine level: A_1[B, nbr_s] = sum_{i in B} sum_{j in nbr_s} P0[i]^T A_ij P0[j].
// One CTA per (box, slot) pair; rows of B in chunks of 32; entries of a row are sorted by
// window index, so the slot's entries form one contiguous run found by binary search.
constexpr int kRapRows = 32;
__global__ void __launch_bounds__(256) k_rap_fine(
    const int64_t* __restrict__ pair_box, const int64_t* __restrict__ nbr_ptr, const int64_t* __restrict__ nbr,
    const int32_t* __restrict__ win_off, const int64_t* __restrict__ slot_src, const int32_t* __restrict__ win_size,
    const int64_t* __restrict__ box_row, const int64_t* __restrict__ row_ptr,
    const uint16_t* __restrict__ idx, const double* __restrict__ vals, const double* __restrict__ P0, int b,
    int64_t npairs, const int64_t* __restrict__ row_ptr1, double* __restrict__ vals1) {
  extern __shared__ double sm[];
  double* Pi = sm;                       // kRapRows x b
  double* Wi = sm + kRapRows * b;        // kRapRows x b
  __shared__ int64_t kr[kRapRows][2];
  const int bb = b * b;
  for (int64_t e = blockIdx.x; e < npairs; e += gridDim.x) {
    const int64_t B = pair_box[e];
    const int s = (int)(e - nbr_ptr[B]);
    // the slot's window run: tree rows [slot_src[e], slot_src[e] + w1 - w0) of the neighbour box
    const int w0 = win_off[e];
    const int64_t cstart = slot_src[e];
    const int w1 = (e + 1 < nbr_ptr[B + 1]) ? win_off[e + 1] : win_size[B];
    double acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.0;
    const int64_t r0 = box_row[B], r1 = box_row[B + 1];
    for (int64_t rc = r0; rc < r1; rc += kRapRows) {
      const int nr = (int)((r1 - rc) < kRapRows ? (r1 - rc) : kRapRows);
      if (threadIdx.x < nr) {
        const int64_t row = rc + threadIdx.x;
        // entries are sorted by window index; padding repeats the last index with value 0
        const int64_t lo = row_ptr[row], end = row_ptr[row + 1];
        int64_t a = lo, z = end;
        while (a < z) { const int64_t m = (a + z) >> 1; if (idx[m] < w0) a = m + 1; else z = m; }
        int64_t a2 = a, z2 = end;
        while (a2 < z2) { const int64_t m = (a2 + z2) >> 1; if (idx[m] < w1) a2 = m + 1; else z2 = m; }
        kr[threadIdx.x][0] = a;
        kr[threadIdx.x][1] = a2;
      }
      for (int t = threadIdx.x; t < nr * b; t += blockDim.x) Pi[t] = P0[(rc + t / b) * b + t % b];
      __syncthreads();
      for (int t = threadIdx.x; t < nr * b; t += blockDim.x) {
        const int rr = t / b, q = t % b;
        double w = 0.0;
        for (int64_t k = kr[rr][0]; k < kr[rr][1]; ++k)
          w += vals[k] * P0[(cstart + (idx[k] - w0)) * b + q];
        Wi[t] = w;
      }
      __syncthreads();
      for (int u = 0; u < 16; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        if (t < bb) {
          const int qp = t / b, q = t % b;
          double sacc = 0.0;
          for (int rr = 0; rr < nr; ++rr) sacc += Pi[rr * b + qp] * Wi[rr * b + q];
          acc[u] += sacc;
        }
      }
      __syncthreads();
    }
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < bb) {
        const int qp = t / b, q = t % b;
        vals1[row_ptr1[B * b + qp] + (int64_t)s * b + q] = acc[u];
      }
    }
  }
}

// Galerkin product between agglomerated levels: A_{l+1}[B, B'] = sum over children c of B,
// c' of B' adjacent on level l, of P~_c^T A_l[c, c'] P~_{c'}.  One CTA per (B, slot) pair.
__global__ void __launch_bounds__(256) k_rap_coarse(
    const int64_t* __restrict__ pair_box, const int64_t* __restrict__ nbr_ptr1, const int64_t* __restrict__ nbr1,
    const int64_t* __restrict__ nbr_ptr0, const int64_t* __restrict__ nbr0, const int64_t* __restrict__ row_ptr0,
    const double* __restrict__ vals0, const double* __restrict__ Pt, int b, int fan, int64_t npairs,
    const int64_t* __restrict__ row_ptr1, double* __restrict__ vals1) {
  extern __shared__ double sm[];
  const int bb = b * b;
  double* Ab = sm;          // A_l[c, c'] block
  double* Pc2 = sm + bb;    // P~_{c'}
  double* Mb = sm + 2 * bb; // A_l[c,c'] P~_{c'}
  double* Pc = sm + 3 * bb; // P~_c
  for (int64_t e = blockIdx.x; e < npairs; e += gridDim.x) {
    const int64_t B = pair_box[e];
    const int s = (int)(e - nbr_ptr1[B]);
    const int64_t Bp = nbr1[e];
    double acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.0;
    for (int64_t c = B * fan; c < (B + 1) * fan; ++c) {
      for (int t = threadIdx.x; t < bb; t += blockDim.x) Pc[t] = Pt[c * bb + t];
      for (int64_t f = nbr_ptr0[c]; f < nbr_ptr0[c + 1]; ++f) {
        const int64_t cp = nbr0[f];
        if (cp / fan != Bp) continue;
        const int64_t slot = f - nbr_ptr0[c];
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
          const int qp = t / b, q = t % b;
          Ab[t] = vals0[row_ptr0[c * b + qp] + slot * b + q];
          Pc2[t] = Pt[cp * bb + t];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
          const int qp = t / b, q = t % b;
          double m = 0.0;
          for (int k = 0; k < b; ++k) m += Ab[qp * b + k] * Pc2[k * b + q];
          Mb[t] = m;
        }
        __syncthreads();
        for (int u = 0; u < 16; ++u) {
          const int t = threadIdx.x + u * blockDim.x;
          if (t < bb) {
            const int qp = t / b, q = t % b;
            double m = 0.0;
            for (int k = 0; k < b; ++k) m += Pc[k * b + qp] * Mb[k * b + q];
            acc[u] += m;
          }
        }
      }
      __syncthreads();
    }
    for (int u = 0; u < 16; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < bb) {
        const int qp = t / b, q = t % b;
        vals1[row_ptr1[B * b + qp] + (int64_t)s * b + q] = acc[u];
      }
    }
  }
}

// Dense copy of the boxes [B0, B0 + nbox) of a block level (coarsest of one problem):
// D[(B,q'), (nbr_s, q)] = block value, rows and columns relative to box B0.
__global__ void k_blocks_to_dense(const int64_t* __restrict__ nbr_ptr, const int64_t* __restrict__ nbr,
                                  const int64_t* __restrict__ row_ptr, const double* __restrict__ vals, int64_t nbox,
                                  int b, double* D, int64_t ld, int64_t B0) {
  const int64_t nc = nbox * b;
  for (int64_t rl = blockIdx.x; rl < nc; rl += gridDim.x) {
    const int64_t r = B0 * b + rl;
    const int64_t B = r / b;
    const int64_t e0 = nbr_ptr[B], nn = nbr_ptr[B + 1] - e0;
    for (int64_t t = threadIdx.x; t < nn * b; t += blockDim.x) {
      const int64_t s = t / b;
      const int q = (int)(t - s * b);
      D[rl * ld + (nbr[e0 + s] - B0) * b + q] = vals[row_ptr[r] + t];
    }
  }
}

// Block values of a level in the export layout ((pair, q', q) contiguous).
__global__ void k_blocks_export(const int64_t* __restrict__ pair_box, const int64_t* __restrict__ nbr_ptr,
                                const int64_t* __restrict__ row_ptr, const double* __restrict__ vals, int64_t npairs,
                                int b, double* out) {
  const int bb = b * b;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npairs * bb; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / bb;
    const int rem = (int)(t - e * bb);
    const int qp = rem / b, q = rem % b;
    const int64_t B = pair_box[e];
    const int64_t s = e - nbr_ptr[B];
    out[t] = vals[row_ptr[B * b + qp] + s * b + q];
  }
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ a, D* __restrict__ o, int64_t m) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    o[k] = (D)a[k];
}

// splitmix64 (Steele, Lea, Flood 2014): value number `ctr` of the sequence seeded by `seed`,
// mapped to [-1, 1).  Counter-based, so any index can be generated independently.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Lanczos start vector: v[k] = U(seed, label(k)), label = caller index on the fine level.
__global__ void k_splitmix_vec(uint64_t seed, const int64_t* __restrict__ label, double* v, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v[k] = splitmix_uniform(seed, (uint64_t)(label ? label[k] : k));
}

}  // namespace r3mg
