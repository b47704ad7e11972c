// FP64 Rayleigh-Ritz on the small LOBPCG pencil (Sec. II.B, operation 4).
//
// The paper solves the O(J_K) Rayleigh-Ritz problem sequentially on each
// processor.  Here one CTA per element does it in FP64, all elements of a
// batch at once:
//   1. symmetrise A and B (Gram blocks are computed for the upper block
//      triangle), equilibrate by D = diag(B)^-1/2;
//   2. Cholesky B = L L^T, with a pivot-ratio condition check; when it fails
//      with P present the pencil is rebuilt without P (the usual LOBPCG
//      restart), otherwise the element is flagged;
//   3. C = L^-1 A L^-T by two triangular solves;
//   4. Householder tridiagonalisation of C;
//   5. the lowest m eigenvalues by Sturm-sequence bisection, one thread each;
//   6. eigenvectors of the tridiagonal matrix by inverse iteration with
//      partial-pivoting elimination, re-orthogonalised inside clusters of
//      close eigenvalues (modified Gram-Schmidt);
//   7. back-transformation by the Householder reflectors, Y = D L^-T Z.
// Every loop is bounded by the matrix size; nothing waits on another CTA.
#include <cfloat>

#include "internal.h"

namespace dgdft {

namespace {

constexpr int RR_THREADS = 256;

struct RRWork {
  double *L, *C, *H, *Z, *d, *e, *scal, *lam, *ptmp, *tri;
  int* cstart;
};

__device__ RRWork carve(double* w, int n, int m) {
  RRWork r;
  r.L = w;
  r.C = r.L + (size_t)n * n;
  r.H = r.C + (size_t)n * n;
  r.Z = r.H + (size_t)n * n;
  r.d = r.Z + (size_t)n * m;
  r.e = r.d + n;
  r.scal = r.e + n;
  r.lam = r.scal + n;
  r.ptmp = r.lam + m;
  r.tri = r.ptmp + n;                       // 5 n per eigenvector slot
  r.cstart = reinterpret_cast<int*>(r.tri + (size_t)5 * n * m);
  return r;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

__device__ double block_min(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = fmin(s, red[w]);
  return s;
}

__device__ double block_max(double v, double* red) { return -block_min(-v, red); }

// Number of eigenvalues of the tridiagonal (d, e) below x.
__device__ int sturm_count(const double* d, const double* e, int n, double x, double tiny) {
  int c = 0;
  double q = 1.0;
  for (int i = 0; i < n; ++i) {
    const double off = (i > 0) ? e[i - 1] * e[i - 1] / q : 0.0;
    q = d[i] - x - off;
    if (fabs(q) < tiny) q = -tiny;
    if (q < 0.0) ++c;
  }
  return c;
}

// Solve (T - lam I) x = b in place (b -> x) by Gaussian elimination with
// partial pivoting; u0/u1/u2/mul are n-long scratch vectors.
__device__ void tri_solve(const double* d, const double* e, int n, double lam, double* b, double* u0,
                          double* u1, double* u2, double* mul, double eps) {
  for (int i = 0; i < n; ++i) {
    u0[i] = d[i] - lam;
    u1[i] = (i < n - 1) ? e[i] : 0.0;
    u2[i] = 0.0;
  }
  for (int i = 0; i < n - 1; ++i) {
    const double sub = e[i];
    if (fabs(sub) > fabs(u0[i])) {
      // swap rows i and i+1
      const double r0a = sub, r0b = u0[i + 1], r0c = (i + 1 < n - 1) ? u1[i + 1] : 0.0;
      const double r1a = u0[i], r1b = u1[i], r1c = u2[i];
      u0[i] = r0a;
      u1[i] = r0b;
      u2[i] = r0c;
      const double mlt = r1a / r0a;
      u0[i + 1] = r1b - mlt * r0b;
      u1[i + 1] = r1c - mlt * r0c;
      const double t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t - mlt * b[i + 1];
      mul[i] = mlt;
    } else {
      if (u0[i] == 0.0) u0[i] = eps;
      const double mlt = sub / u0[i];
      u0[i + 1] -= mlt * u1[i];
      b[i + 1] -= mlt * b[i];
      mul[i] = mlt;
    }
  }
  for (int i = 0; i < n; ++i)
    if (fabs(u0[i]) < eps) u0[i] = (u0[i] >= 0.0) ? eps : -eps;
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    if (i + 1 < n) s -= u1[i] * b[i + 1];
    if (i + 2 < n) s -= u2[i] * b[i + 2];
    b[i] = s / u0[i];
  }
}

__device__ __forceinline__ double hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (double)(h & 0xFFFFFF) / (double)0x800000 - 1.0;
}

__global__ void __launch_bounds__(RR_THREADS) rr_kernel(const RRTask* __restrict__ tasks) {
  const RRTask T = tasks[blockIdx.x];
  if (T.state && !T.state[ST_ACTIVE]) return;
  __shared__ double red[32];
  __shared__ int sflag;
  __shared__ double sval[4];
  const int m = T.m;
  int n = (T.mode == RR_FIXED) ? T.n_fixed
          : (T.mode == RR_INITIAL) ? m
          : (T.state[ST_HAS_P] ? 3 * m : 2 * m);
  const int bm = (T.mode == RR_FIXED) ? n : m;  // symmetrisation block size
  const int n_out = (T.mode == RR_LOBPCG) ? 3 * m : n;
  bool dropped = false;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (;;) {
    RRWork W = carve(T.work, n, m);
    // 1. symmetrise and equilibrate
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      const int br = r / bm, bc = c / bm;
      double a, b;
      if (br < bc) {
        a = T.A[r + (size_t)c * T.ld];
        b = T.B[r + (size_t)c * T.ld];
      } else if (br > bc) {
        a = T.A[c + (size_t)r * T.ld];
        b = T.B[c + (size_t)r * T.ld];
      } else {
        a = 0.5 * (T.A[r + (size_t)c * T.ld] + T.A[c + (size_t)r * T.ld]);
        b = 0.5 * (T.B[r + (size_t)c * T.ld] + T.B[c + (size_t)r * T.ld]);
      }
      W.L[idx] = b;
      W.C[idx] = a;
    }
    if (tid == 0) sflag = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      const double bii = W.L[i + (size_t)i * n];
      if (!(bii > 0.0) || !isfinite(bii)) {
        sflag = 1;
        W.scal[i] = 0.0;
      } else {
        W.scal[i] = 1.0 / sqrt(bii);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      const double s = W.scal[r] * W.scal[c];
      W.L[idx] *= s;
      W.C[idx] *= s;
    }
    __syncthreads();
    // 2. Cholesky, lower triangle, column-major
    double pmin = DBL_MAX, pmax = 0.0;
    for (int k = 0; k < n && !sflag; ++k) {
      if (tid == 0) {
        const double p = W.L[k + (size_t)k * n];
        if (!(p > 0.0) || !isfinite(p)) {
          sflag = 1;
        } else {
          const double dk = sqrt(p);
          W.L[k + (size_t)k * n] = dk;
          sval[0] = dk;
        }
      }
      __syncthreads();
      if (sflag) break;
      const double dk = sval[0];
      pmin = fmin(pmin, dk);
      pmax = fmax(pmax, dk);
      for (int i = k + 1 + tid; i < n; i += nt) W.L[i + (size_t)k * n] /= dk;
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * nk; t += nt) {
        const int jj = t / nk, ii = t - jj * nk;
        if (ii < jj) continue;
        const int i = k + 1 + ii, j = k + 1 + jj;
        W.L[i + (size_t)j * n] -= W.L[i + (size_t)k * n] * W.L[j + (size_t)k * n];
      }
      __syncthreads();
    }
    bool fail = sflag != 0;
    if (!fail && (pmax / pmin) * (pmax / pmin) > T.cond_max) fail = true;
    __syncthreads();
    if (fail) {
      if (T.mode == RR_LOBPCG && n == 3 * m) {
        n = 2 * m;
        dropped = true;
        __syncthreads();
        continue;
      }
      if (tid == 0 && T.state) {
        T.state[ST_ERROR] |= ERR_CHOL;
        T.state[ST_ACTIVE] = 0;
      }
      if (tid == 0 && !T.state) T.theta[0] = __longlong_as_double(0x7ff8000000000000LL);
      return;
    }
    // 3. C = L^-1 A L^-T
    for (int c = tid; c < n; c += nt) {
      double* col = W.C + (size_t)c * n;
      for (int i = 0; i < n; ++i) {
        double s0 = col[i], s1 = 0.0;
        int k = 0;
        for (; k + 1 < i; k += 2) {
          s0 -= W.L[i + (size_t)k * n] * col[k];
          s1 -= W.L[i + (size_t)(k + 1) * n] * col[k + 1];
        }
        for (; k < i; ++k) s0 -= W.L[i + (size_t)k * n] * col[k];
        col[i] = (s0 + s1) / W.L[i + (size_t)i * n];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      W.H[c + (size_t)r * n] = W.C[idx];
    }
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
      double* col = W.H + (size_t)c * n;
      for (int i = 0; i < n; ++i) {
        double s0 = col[i], s1 = 0.0;
        int k = 0;
        for (; k + 1 < i; k += 2) {
          s0 -= W.L[i + (size_t)k * n] * col[k];
          s1 -= W.L[i + (size_t)(k + 1) * n] * col[k + 1];
        }
        for (; k < i; ++k) s0 -= W.L[i + (size_t)k * n] * col[k];
        col[i] = (s0 + s1) / W.L[i + (size_t)i * n];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      W.C[idx] = 0.5 * (W.H[idx] + W.H[c + (size_t)r * n]);
    }
    __syncthreads();
    // 4. Householder tridiagonalisation; reflector k in column k of H
    for (int idx = tid; idx < n * n; idx += nt) W.H[idx] = 0.0;
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
      double part = 0.0;
      for (int i = k + 1 + tid; i < n; i += nt) {
        const double x = W.C[i + (size_t)k * n];
        part += x * x;
      }
      const double xx = block_sum(part, red);
      const double x0 = W.C[k + 1 + (size_t)k * n];
      const double alpha = (x0 >= 0.0) ? -sqrt(xx) : sqrt(xx);
      const double vn2 = xx - 2.0 * alpha * x0 + alpha * alpha;
      if (tid == 0) {
        W.d[k] = W.C[k + (size_t)k * n];
        W.e[k] = (vn2 > 0.0) ? alpha : x0;
      }
      if (!(vn2 > 0.0)) {
        __syncthreads();
        continue;
      }
      const double inv = 1.0 / sqrt(vn2);
      double* v = W.H + (size_t)k * n;
      for (int i = k + 1 + tid; i < n; i += nt)
        v[i] = (i == k + 1 ? x0 - alpha : W.C[i + (size_t)k * n]) * inv;
      __syncthreads();
      // p = C22 v: one warp per row
      const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
      for (int i = k + 1 + warp; i < n; i += nw) {
        double s = 0.0;
        for (int j = k + 1 + lane; j < n; j += 32) s += W.C[j + (size_t)i * n] * v[j];
        s = warp_sum(s);
        if (lane == 0) W.ptmp[i] = s;
      }
      __syncthreads();
      double kp = 0.0;
      for (int i = k + 1 + tid; i < n; i += nt) kp += v[i] * W.ptmp[i];
      const double K = block_sum(kp, red);
      for (int i = k + 1 + tid; i < n; i += nt) W.ptmp[i] = 2.0 * W.ptmp[i] - 2.0 * K * v[i];
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * nk; t += nt) {
        const int jj = t / nk, ii = t - jj * nk;
        const int i = k + 1 + ii, j = k + 1 + jj;
        W.C[i + (size_t)j * n] -= v[i] * W.ptmp[j] + W.ptmp[i] * v[j];
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        W.d[n - 2] = W.C[n - 2 + (size_t)(n - 2) * n];
        W.e[n - 2] = W.C[n - 1 + (size_t)(n - 2) * n];
      }
      W.d[n - 1] = W.C[n - 1 + (size_t)(n - 1) * n];
      W.e[n - 1] = 0.0;
    }
    __syncthreads();
    // 5. bisection for the lowest m eigenvalues
    double glo = DBL_MAX, ghi = -DBL_MAX, gnorm = 0.0;
    for (int i = tid; i < n; i += nt) {
      const double r = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(W.e[i]) : 0.0);
      glo = fmin(glo, W.d[i] - r);
      ghi = fmax(ghi, W.d[i] + r);
      gnorm = fmax(gnorm, fabs(W.d[i]) + r);
    }
    glo = block_min(glo, red);
    ghi = block_max(ghi, red);
    gnorm = block_max(gnorm, red);
    const double eps = DBL_EPSILON;
    const double tiny = DBL_MIN / eps;
    const double pad = 2.0 * eps * fmax(gnorm, 1e-300) * n;
    glo -= pad;
    ghi += pad;
    for (int i = tid; i < m; i += nt) {
      double lo = glo, hi = ghi;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi) || hi - lo <= 4.0 * eps * fmax(fabs(lo), fabs(hi))) break;
        if (sturm_count(W.d, W.e, n, mid, tiny) > i)
          hi = mid;
        else
          lo = mid;
      }
      W.lam[i] = 0.5 * (lo + hi);
    }
    __syncthreads();
    // 6. inverse iteration, clusters re-orthogonalised
    const double ortol = 1e-3 * gnorm;
    if (tid == 0) {
      for (int i = 0; i < m; ++i)
        W.cstart[i] = (i == 0 || W.lam[i] - W.lam[i - 1] > ortol) ? i : W.cstart[i - 1];
    }
    __syncthreads();
    const double sep = 10.0 * eps * gnorm;
    for (int s = tid; s < m; s += nt) {
      if (W.cstart[s] != s) continue;
      double lam_prev = -DBL_MAX;
      for (int q = s; q < m && W.cstart[q] == s; ++q) {
        double lam = W.lam[q];
        if (q > s && lam - lam_prev < sep) lam = lam_prev + sep;
        lam_prev = lam;
        double* b = W.Z + (size_t)q * n;
        double* u0 = W.tri + (size_t)5 * n * q;
        double* u1 = u0 + n;
        double* u2 = u1 + n;
        double* mul = u2 + n;
        for (int i = 0; i < n; ++i) b[i] = hash_unit(i, q + 7919u * blockIdx.x);
        for (int it = 0; it < 4; ++it) {
          double nb = 0.0;
          for (int i = 0; i < n; ++i) nb += b[i] * b[i];
          nb = 1.0 / sqrt(nb);
          for (int i = 0; i < n; ++i) b[i] *= nb;
          tri_solve(W.d, W.e, n, lam, b, u0, u1, u2, mul, eps * fmax(gnorm, 1e-300));
          for (int p = s; p < q; ++p) {
            const double* zp = W.Z + (size_t)p * n;
            double dp = 0.0;
            for (int i = 0; i < n; ++i) dp += zp[i] * b[i];
            for (int i = 0; i < n; ++i) b[i] -= dp * zp[i];
          }
        }
        double nb = 0.0;
        for (int i = 0; i < n; ++i) nb += b[i] * b[i];
        nb = 1.0 / sqrt(nb);
        for (int i = 0; i < n; ++i) b[i] *= nb;
      }
    }
    __syncthreads();
    // 7. back-transformation by the reflectors, then Y = D L^-T Z
    for (int k = n - 3; k >= 0; --k) {
      const double* v = W.H + (size_t)k * n;
      const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
      for (int c = warp; c < m; c += nw) {
        const double* zc = W.Z + (size_t)c * n;
        double s = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) s += v[i] * zc[i];
        s = warp_sum(s);
        if (lane == 0) W.ptmp[c] = s;
      }
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * m; t += nt) {
        const int c = t / nk, i = k + 1 + (t - c * nk);
        W.Z[i + (size_t)c * n] -= 2.0 * v[i] * W.ptmp[c];
      }
      __syncthreads();
    }
    for (int c = tid; c < m; c += nt) {
      double* zc = W.Z + (size_t)c * n;
      for (int i = n - 1; i >= 0; --i) {
        double s = zc[i];
        for (int k = i + 1; k < n; ++k) s -= W.L[k + (size_t)i * n] * zc[k];
        zc[i] = s / W.L[i + (size_t)i * n];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n_out * m; idx += nt) {
      const int r = idx % n_out, c = idx / n_out;
      T.Y[r + (size_t)c * T.ldy] = (r < n) ? W.Z[r + (size_t)c * n] * W.scal[r] : 0.0;
    }
    for (int c = tid; c < m; c += nt) T.theta[c] = W.lam[c];
    if (tid == 0 && dropped && T.state) T.state[ST_FALLBACK] += 1;
    return;
  }
}

}  // namespace

size_t rr_work_doubles(int n_max, int m) {
  return (size_t)3 * n_max * n_max + (size_t)n_max * m + 4 * (size_t)n_max + m + (size_t)5 * n_max * m +
         (size_t)m + 16;
}

void launch_rr(const RRTask* d_tasks, int ntask, cudaStream_t st) {
  if (ntask <= 0) return;
  rr_kernel<<<ntask, RR_THREADS, 0, st>>>(d_tasks);
}

}  // namespace dgdft
