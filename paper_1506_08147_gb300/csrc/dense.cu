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
  double *L, *C, *H, *Z, *d, *e, *scal, *lam, *ptmp, *tri, *shift;
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
  r.shift = r.tri + (size_t)5 * n * m;
  r.cstart = reinterpret_cast<int*>(r.shift + m);
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

// Number of eigenvalues of the tridiagonal (d, e) below x, in FP32 (used to
// locate shifts; FP64 is ~60x slower per operation on this part).
__device__ int sturm_count_f(const float* d, const float* e2, int n, float x, float tiny) {
  int c = 0;
  float q = 1.0f;
  for (int i = 0; i < n; ++i) {
    q = d[i] - x - ((i > 0) ? __fdividef(e2[i - 1], q) : 0.0f);
    if (fabsf(q) < tiny) q = -tiny;
    if (q < 0.0f) ++c;
  }
  return c;
}

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

// Eigenvectors of the symmetric tridiagonal (d, e) for the m lowest
// eigenvalue estimates lam[] by inverse iteration, all vectors at once
// (thread q owns vector q, column q of Z).  Estimates closer than ortol form
// clusters: their shifts are kept at least 10 eps |T| apart and after every
// step the cluster's vectors are orthogonalised by modified Gram-Schmidt
// (inverse iteration alone cannot separate them).  Isolated vectors take
// the Rayleigh quotient as the shift after the first step (cubic
// convergence from a rough start).  The estimates come from bisection whose
// location error can approach ortol, so two close eigenvalues taken as
// isolated may both converge to one eigenvector; the vectors are therefore
// checked against their next few neighbours, and if any two overlap the
// inverse iteration is redone with all m vectors in one orthogonalised
// cluster (rare, and then ~m^2 n more work).  On return the columns are
// orthonormal and lam[] holds their Rayleigh quotients.  shift, dots: m
// doubles; tri: 5 n doubles per vector; cstart: m ints.  Every thread of the
// block calls.
__device__ void tri_eigvecs(const double* d, const double* e, int n, int m, double* lam, double* Z, int ldz,
                            int* cstart, double* shift, double* dots, double* tri, double ortol, double gnorm,
                            double* red, unsigned seed) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const double eps = DBL_EPSILON;
  const double sep = 10.0 * eps * fmax(gnorm, 1e-300);
  __shared__ int any_cluster, overlap;
  if (tid == 0) {
    any_cluster = 0;
    for (int i = 0; i < m; ++i) {
      const bool joins = i > 0 && lam[i] - lam[i - 1] <= ortol;
      cstart[i] = joins ? cstart[i - 1] : i;
      shift[i] = joins ? fmax(lam[i], shift[i - 1] + sep) : lam[i];
      any_cluster |= joins;
    }
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
  for (int it = 0; it < 3; ++it) {
    for (int q = tid; q < m; q += nt) {
      double* b = Z + (size_t)q * ldz;
      double* u0 = tri + (size_t)5 * n * q;
      const bool single = cstart[q] == q && (q + 1 >= m || cstart[q + 1] != q);
      if (it == 0)
        for (int i = 0; i < n; ++i) b[i] = hash_unit(i, q + 7919u * seed);
      double lq = shift[q];
      if (single && it > 0) {
        double rq = 0.0;
        for (int i = 0; i < n; ++i) {
          double t = d[i] * b[i];
          if (i > 0) t += e[i - 1] * b[i - 1];
          if (i + 1 < n) t += e[i] * b[i + 1];
          rq += b[i] * t;
        }
        lq = rq;
      }
      tri_solve(d, e, n, lq, b, u0, u0 + n, u0 + 2 * n, u0 + 3 * n, eps * fmax(gnorm, 1e-300));
      double nb = 0.0;
      for (int i = 0; i < n; ++i) nb += b[i] * b[i];
      nb = 1.0 / sqrt(nb);
      for (int i = 0; i < n; ++i) b[i] *= nb;
    }
    __syncthreads();
    if (!any_cluster) continue;
    for (int j = 0; j < m; ++j) {
      const bool clustered = (cstart[j] != j) || (j + 1 < m && cstart[j + 1] == cstart[j]);
      if (!clustered) continue;  // uniform across the block
      double* zj = Z + (size_t)j * ldz;
      double part = 0.0;
      for (int i = tid; i < n; i += nt) part += zj[i] * zj[i];
      const double inv = 1.0 / sqrt(block_sum(part, red));
      for (int i = tid; i < n; i += nt) zj[i] *= inv;
      __syncthreads();
      int kend = j + 1;
      while (kend < m && cstart[kend] == cstart[j]) ++kend;
      for (int k = j + 1 + warp; k < kend; k += nw) {
        const double* zk = Z + (size_t)k * ldz;
        double s2 = 0.0;
        for (int i = lane; i < n; i += 32) s2 += zj[i] * zk[i];
        s2 = warp_sum(s2);
        if (lane == 0) dots[k] = s2;
      }
      __syncthreads();
      const int rest = kend - j - 1;
      for (int t = tid; t < rest * n; t += nt) {
        const int k = j + 1 + t / n, i = t - (k - j - 1) * n;
        Z[i + (size_t)k * ldz] -= dots[k] * zj[i];
      }
      __syncthreads();
    }
  }
  if (pass == 1) break;
  // overlap check: unit vectors of distinct eigenvalues are orthogonal to
  // rounding; a large product means two of them found the same eigenvector
  constexpr int REACH = 4;
  if (tid == 0) overlap = 0;
  __syncthreads();
  for (int t = warp; t < m * REACH; t += nw) {
    const int j = t / REACH, k = j + 1 + (t - j * REACH);
    if (k >= m) continue;
    const double* zj = Z + (size_t)j * ldz;
    const double* zk = Z + (size_t)k * ldz;
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 += zj[i] * zk[i];
    s2 = warp_sum(s2);
    if (lane == 0 && fabs(s2) > 1e-3) overlap = 1;
  }
  __syncthreads();
  if (!overlap) break;
  if (tid == 0) {
    any_cluster = 1;
    for (int i = 1; i < m; ++i) {
      cstart[i] = 0;
      shift[i] = fmax(shift[i], shift[i - 1] + sep);
    }
  }
  __syncthreads();
  }
  // eigenvalues as FP64 Rayleigh quotients z^T T z of the unit vectors
  for (int j = warp; j < m; j += nw) {
    const double* zj = Z + (size_t)j * ldz;
    double s5 = 0.0;
    for (int i = lane; i < n; i += 32) {
      double t = d[i] * zj[i];
      if (i > 0) t += e[i - 1] * zj[i - 1];
      if (i + 1 < n) t += e[i] * zj[i + 1];
      s5 += zj[i] * t;
    }
    s5 = warp_sum(s5);
    if (lane == 0) lam[j] = s5;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RR_THREADS) rr_kernel(const RRTask* __restrict__ tasks) {
  const RRTask T = tasks[blockIdx.x];
  if (T.state && !T.state[ST_ACTIVE]) return;
  if (T.state && (T.state[ST_ERROR] & ERR_TIMEOUT)) {
    // a wait in this iteration's Gram launch ran out: its products are stale
    if (threadIdx.x == 0) T.state[ST_ACTIVE] = 0;
    return;
  }
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
    // the last LOBPCG resort (X alone) takes any positive-definite B: its
    // Rayleigh-Ritz re-orthonormalises a block that has drifted
    const bool last_resort = T.mode == RR_LOBPCG && n == m;
    const double cond_lim = last_resort ? (T.restart_max > 0 ? 1e6 : 1e300) : T.cond_max;
    if (!fail && (pmax / pmin) * (pmax / pmin) > cond_lim) fail = true;
    // read before the barrier: thread 0 updates the count after it
    const bool can_restart =
        T.mode == RR_LOBPCG && T.restart_max > 0 && T.state && T.state[ST_NRESTART] < T.restart_max;
    __syncthreads();
    if (fail) {
      if (T.mode == RR_LOBPCG && n == 3 * m) {
        n = 2 * m;
        dropped = true;
        __syncthreads();
        continue;
      }
      if (T.mode == RR_LOBPCG && n == 2 * m) {
        // [X W] is numerically dependent too (W nearly inside span X or
        // its columns nearly parallel): Rayleigh-Ritz on X alone, a
        // rotation of the current block; the next iteration brings a new W
        n = m;
        dropped = true;
        __syncthreads();
        continue;
      }
      if (can_restart) {
        // no usable pencil, not even X alone: keep X (Y = [I; 0]) and let
        // the restart step perturb it and drop P (Ritz values unchanged)
        const int nr = 3 * m;
        for (int idx = tid; idx < nr * m; idx += nt) {
          const int r = idx % nr, c = idx / nr;
          const double y = (r == c) ? 1.0 : 0.0;
          T.Y[r + (size_t)c * T.ldy] = y;
          if (T.Yf) T.Yf[r + (size_t)c * T.ldy] = (float)y;
        }
        if (tid == 0) {
          T.state[ST_RESTART] = 1;
          T.state[ST_NRESTART] += 1;
          T.state[ST_FALLBACK] += 1;
        }
        return;
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
    // 6. eigenvectors of the tridiagonal by inverse iteration
    tri_eigvecs(W.d, W.e, n, m, W.lam, W.Z, n, W.cstart, W.shift, W.ptmp, W.tri, 1e-7 * gnorm, gnorm, red,
                blockIdx.x);
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
      const double y = (r < n) ? W.Z[r + (size_t)c * n] * W.scal[r] : 0.0;
      T.Y[r + (size_t)c * T.ldy] = y;
      if (T.Yf) T.Yf[r + (size_t)c * T.ldy] = (float)y;
    }
    for (int c = tid; c < m; c += nt) T.theta[c] = W.lam[c];
    if (tid == 0 && dropped && T.state) T.state[ST_FALLBACK] += 1;
    return;
  }
}


// Shared-memory variant for pencils whose n x n working matrix and n x m
// eigenvector block fit in one CTA's shared memory (n = 3m <= ~150 at m = 48).
// Same algorithm; every O(n^3) phase runs on shared memory with all threads
// (right-looking triangular solves, in-place Householder reflectors) and the
// eigenvalues are found by parallel multisection of the Sturm count.
constexpr int RRS_THREADS = 512;

__global__ void __launch_bounds__(RRS_THREADS) rr_smem_kernel(const RRTask* __restrict__ tasks) {
  const RRTask T = tasks[blockIdx.x];
  if (T.state && !T.state[ST_ACTIVE]) return;
  if (T.state && (T.state[ST_ERROR] & ERR_TIMEOUT)) {
    // a wait in this iteration's Gram launch ran out: its products are stale
    if (threadIdx.x == 0) T.state[ST_ACTIVE] = 0;
    return;
  }
  extern __shared__ __align__(16) double smd[];
  __shared__ double red[32];
  __shared__ int sflag;
  __shared__ double sval[4];
  const int m = T.m;
  int n = (T.mode == RR_FIXED) ? T.n_fixed
          : (T.mode == RR_INITIAL) ? m
          : (T.state[ST_HAS_P] ? 3 * m : 2 * m);
  const int bm = (T.mode == RR_FIXED) ? n : m;
  const int n_out = (T.mode == RR_LOBPCG) ? 3 * m : n;
  const int nmax = n;  // shared layout is sized for the first attempt
  double* S = smd;                          // n x n working matrix
  double* Z = S + (size_t)nmax * nmax;      // n x m eigenvectors
  double* d = Z + (size_t)nmax * m;         // tridiagonal diagonal
  double* e = d + nmax;                     // off-diagonal
  double* scal = e + nmax;                  // equilibration
  double* ptmp = scal + nmax;               // n scratch
  double* lam = ptmp + nmax;                // m eigenvalues
  double* lo_s = lam + m;                   // m interval bounds
  double* hi_s = lo_s + m;
  int* cnt = reinterpret_cast<int*>(hi_s + m);  // multisection counts (nt)
  bool dropped = false;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  for (;;) {
    RRWork W = carve(T.work, n, m);  // global: L (n x n), tri-solve scratch, cluster starts
    // 1. B: symmetrise, equilibrate, Cholesky in shared memory
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      const int br = r / bm, bc = c / bm;
      double b;
      if (br < bc) b = T.B[r + (size_t)c * T.ld];
      else if (br > bc) b = T.B[c + (size_t)r * T.ld];
      else b = 0.5 * (T.B[r + (size_t)c * T.ld] + T.B[c + (size_t)r * T.ld]);
      S[idx] = b;
    }
    if (tid == 0) sflag = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      const double bii = S[i + (size_t)i * n];
      if (!(bii > 0.0) || !isfinite(bii)) {
        sflag = 1;
        scal[i] = 0.0;
      } else {
        scal[i] = 1.0 / sqrt(bii);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) S[idx] *= scal[idx % n] * scal[idx / n];
    __syncthreads();
    double pmin = DBL_MAX, pmax = 0.0;
    for (int k = 0; k < n && !sflag; ++k) {
      if (tid == 0) {
        const double p = S[k + (size_t)k * n];
        if (!(p > 0.0) || !isfinite(p)) {
          sflag = 1;
        } else {
          sval[0] = sqrt(p);
          S[k + (size_t)k * n] = sval[0];
        }
      }
      __syncthreads();
      if (sflag) break;
      const double dk = sval[0];
      pmin = fmin(pmin, dk);
      pmax = fmax(pmax, dk);
      const double inv = 1.0 / dk;
      for (int i = k + 1 + tid; i < n; i += nt) S[i + (size_t)k * n] *= inv;
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * nk; t += nt) {
        const int jj = t / nk, ii = t - jj * nk;
        if (ii < jj) continue;
        const int i = k + 1 + ii, j = k + 1 + jj;
        S[i + (size_t)j * n] -= S[i + (size_t)k * n] * S[j + (size_t)k * n];
      }
      __syncthreads();
    }
    bool fail = sflag != 0;
    // the last LOBPCG resort (X alone) takes any positive-definite B: its
    // Rayleigh-Ritz re-orthonormalises a block that has drifted
    const bool last_resort = T.mode == RR_LOBPCG && n == m;
    const double cond_lim = last_resort ? (T.restart_max > 0 ? 1e6 : 1e300) : T.cond_max;
    if (!fail && (pmax / pmin) * (pmax / pmin) > cond_lim) fail = true;
    // read before the barrier: thread 0 updates the count after it
    const bool can_restart =
        T.mode == RR_LOBPCG && T.restart_max > 0 && T.state && T.state[ST_NRESTART] < T.restart_max;
    __syncthreads();
    if (fail) {
      if (T.mode == RR_LOBPCG && n == 3 * m) {
        n = 2 * m;
        dropped = true;
        __syncthreads();
        continue;
      }
      if (T.mode == RR_LOBPCG && n == 2 * m) {
        // [X W] is numerically dependent too (W nearly inside span X or
        // its columns nearly parallel): Rayleigh-Ritz on X alone, a
        // rotation of the current block; the next iteration brings a new W
        n = m;
        dropped = true;
        __syncthreads();
        continue;
      }
      if (can_restart) {
        // no usable pencil, not even X alone: keep X (Y = [I; 0]) and let
        // the restart step perturb it and drop P (Ritz values unchanged)
        const int nr = 3 * m;
        for (int idx = tid; idx < nr * m; idx += nt) {
          const int r = idx % nr, c = idx / nr;
          const double y = (r == c) ? 1.0 : 0.0;
          T.Y[r + (size_t)c * T.ldy] = y;
          if (T.Yf) T.Yf[r + (size_t)c * T.ldy] = (float)y;
        }
        if (tid == 0) {
          T.state[ST_RESTART] = 1;
          T.state[ST_NRESTART] += 1;
          T.state[ST_FALLBACK] += 1;
        }
        return;
      }
      if (tid == 0 && T.state) {
        T.state[ST_ERROR] |= ERR_CHOL;
        T.state[ST_ACTIVE] = 0;
      }
      if (tid == 0 && !T.state) T.theta[0] = __longlong_as_double(0x7ff8000000000000LL);
      return;
    }
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      const double l = (r >= c) ? S[idx] : 0.0;
      W.L[idx] = l;                    // L, column-major
      W.H[c + (size_t)r * n] = l;      // L^T, for the final back-substitution
    }
    __syncthreads();
    // 2. C = L^-1 A L^-T: A into shared memory, two right-looking solves
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      const int br = r / bm, bc = c / bm;
      double a;
      if (br < bc) a = T.A[r + (size_t)c * T.ld];
      else if (br > bc) a = T.A[c + (size_t)r * T.ld];
      else a = 0.5 * (T.A[r + (size_t)c * T.ld] + T.A[c + (size_t)r * T.ld]);
      S[idx] = a * scal[r] * scal[c];
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = 0; k < n; ++k) {
        const double inv = 1.0 / W.L[k + (size_t)k * n];
        for (int c = tid; c < n; c += nt) S[k + (size_t)c * n] *= inv;
        __syncthreads();
        const int nk = n - k - 1;
        for (int t = tid; t < nk * n; t += nt) {
          const int c = t / nk, i = k + 1 + (t - c * nk);
          S[i + (size_t)c * n] -= W.L[i + (size_t)k * n] * S[k + (size_t)c * n];
        }
        __syncthreads();
      }
      if (pass == 0) {  // S <- S^T
        for (int idx = tid; idx < n * n; idx += nt) {
          const int r = idx % n, c = idx / n;
          if (r < c) {
            const double t = S[idx];
            S[idx] = S[c + (size_t)r * n];
            S[c + (size_t)r * n] = t;
          }
        }
        __syncthreads();
      }
    }
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, c = idx / n;
      if (r < c) {
        const double v = 0.5 * (S[idx] + S[c + (size_t)r * n]);
        S[idx] = v;
        S[c + (size_t)r * n] = v;
      }
    }
    __syncthreads();
    // 3. Householder tridiagonalisation; reflector k kept in S[k+1.., k]
    for (int k = 0; k + 2 < n; ++k) {
      double part = 0.0;
      for (int i = k + 1 + tid; i < n; i += nt) {
        const double x = S[i + (size_t)k * n];
        part += x * x;
      }
      const double xx = block_sum(part, red);
      const double x0 = S[k + 1 + (size_t)k * n];
      const double alpha = (x0 >= 0.0) ? -sqrt(xx) : sqrt(xx);
      const double vn2 = xx - 2.0 * alpha * x0 + alpha * alpha;
      if (tid == 0) {
        d[k] = S[k + (size_t)k * n];
        e[k] = (vn2 > 0.0) ? alpha : x0;
      }
      __syncthreads();
      double* v = S + (size_t)k * n;  // column k, rows > k
      if (!(vn2 > 0.0)) {
        for (int i = k + 1 + tid; i < n; i += nt) v[i] = 0.0;
        __syncthreads();
        continue;
      }
      const double inv = 1.0 / sqrt(vn2);
      for (int i = k + 1 + tid; i < n; i += nt) v[i] = (i == k + 1 ? x0 - alpha : v[i]) * inv;
      __syncthreads();
      for (int i = k + 1 + warp; i < n; i += nw) {
        double s2 = 0.0;
        for (int j = k + 1 + lane; j < n; j += 32) s2 += S[j + (size_t)i * n] * v[j];
        s2 = warp_sum(s2);
        if (lane == 0) ptmp[i] = s2;
      }
      __syncthreads();
      double kp = 0.0;
      for (int i = k + 1 + tid; i < n; i += nt) kp += v[i] * ptmp[i];
      const double K = block_sum(kp, red);
      for (int i = k + 1 + tid; i < n; i += nt) ptmp[i] = 2.0 * ptmp[i] - 2.0 * K * v[i];
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * nk; t += nt) {
        const int jj = t / nk, ii = t - jj * nk;
        const int i = k + 1 + ii, j = k + 1 + jj;
        S[i + (size_t)j * n] -= v[i] * ptmp[j] + ptmp[i] * v[j];
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        d[n - 2] = S[n - 2 + (size_t)(n - 2) * n];
        e[n - 2] = S[n - 1 + (size_t)(n - 2) * n];
      }
      d[n - 1] = S[n - 1 + (size_t)(n - 1) * n];
      e[n - 1] = 0.0;
      if (n >= 2) S[n - 1 + (size_t)(n - 2) * n] = 0.0;  // no reflector for the last columns
    }
    __syncthreads();
    // 4. eigenvalue shifts: FP32 Sturm bisection, one thread per eigenvalue
    // (final eigenvalues are FP64 Rayleigh quotients after inverse iteration)
    double glo = DBL_MAX, ghi = -DBL_MAX, gnorm = 0.0;
    for (int i = tid; i < n; i += nt) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      glo = fmin(glo, d[i] - r);
      ghi = fmax(ghi, d[i] + r);
      gnorm = fmax(gnorm, fabs(d[i]) + r);
    }
    glo = block_min(glo, red);
    ghi = block_max(ghi, red);
    gnorm = block_max(gnorm, red);
    const double eps = DBL_EPSILON;
    float* df = reinterpret_cast<float*>(cnt);    // n <= RRS_THREADS floats
    float* ef2 = reinterpret_cast<float*>(ptmp);  // n floats in n doubles
    for (int i = tid; i < n; i += nt) {
      df[i] = (float)d[i];
      ef2[i] = (float)(e[i] * e[i]);
    }
    __syncthreads();
    {
      const float tinyf = 1e-30f;
      const float padf = 1e-6f * (float)fmax(gnorm, 1e-30);
      for (int j = tid; j < m; j += nt) {
        float lo = (float)glo - padf, hi = (float)ghi + padf;
        for (int it = 0; it < 40; ++it) {
          const float mid = 0.5f * (lo + hi);
          if (!(mid > lo && mid < hi)) break;
          if (sturm_count_f(df, ef2, n, mid, tinyf) > j)
            hi = mid;
          else
            lo = mid;
        }
        lam[j] = 0.5 * ((double)lo + (double)hi);
      }
    }
    __syncthreads();
    // 5. eigenvectors by inverse iteration; shifts closer than the FP32
    // location accuracy form clusters, orthogonalised within the cluster
    tri_eigvecs(d, e, n, m, lam, Z, n, W.cstart, lo_s, hi_s, W.tri, 1e-5 * gnorm, gnorm, red, blockIdx.x);
    // 6. back-transformation, then Y = D L^-T Z (right-looking)
    for (int k = n - 3; k >= 0; --k) {
      const double* v = S + (size_t)k * n;
      for (int c = warp; c < m; c += nw) {
        const double* zc = Z + (size_t)c * n;
        double s4 = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) s4 += v[i] * zc[i];
        s4 = warp_sum(s4);
        if (lane == 0) ptmp[c] = s4;
      }
      __syncthreads();
      const int nk = n - k - 1;
      for (int t = tid; t < nk * m; t += nt) {
        const int c = t / nk, i = k + 1 + (t - c * nk);
        Z[i + (size_t)c * n] -= 2.0 * v[i] * ptmp[c];
      }
      __syncthreads();
    }
    for (int i = n - 1; i >= 0; --i) {
      const double inv = 1.0 / W.L[i + (size_t)i * n];
      for (int c = tid; c < m; c += nt) Z[i + (size_t)c * n] *= inv;
      __syncthreads();
      const double* lrow = W.H + (size_t)i * n;  // L[i, k] for k < i, contiguous
      for (int t = tid; t < i * m; t += nt) {
        const int c = t / i, k = t - c * i;
        Z[k + (size_t)c * n] -= lrow[k] * Z[i + (size_t)c * n];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n_out * m; idx += nt) {
      const int r = idx % n_out, c = idx / n_out;
      const double y = (r < n) ? Z[r + (size_t)c * n] * scal[r] : 0.0;
      T.Y[r + (size_t)c * T.ldy] = y;
      if (T.Yf) T.Yf[r + (size_t)c * T.ldy] = (float)y;
    }
    for (int c = tid; c < m; c += nt) T.theta[c] = lam[c];
    if (tid == 0 && dropped && T.state) T.state[ST_FALLBACK] += 1;
    (void)nmax;
    return;
  }
}

}  // namespace

size_t rr_work_doubles(int n_max, int m) {
  return (size_t)3 * n_max * n_max + (size_t)n_max * m + 4 * (size_t)n_max + m + (size_t)5 * n_max * m +
         (size_t)2 * m + 16;
}

size_t rr_smem_bytes(int n, int m) {
  return sizeof(double) * ((size_t)n * n + (size_t)n * m + 4 * (size_t)n + 3 * (size_t)m) +
         sizeof(int) * RRS_THREADS + 64;
}

void init_rr_kernels() { opt_in_dynamic_smem((const void*)rr_smem_kernel); }

// n_max: the largest pencil any task can have (3m for LOBPCG tasks).
void launch_rr(const RRTask* d_tasks, int ntask, cudaStream_t st, int n_max, int m_max, bool dfloat) {
  if (ntask <= 0) return;
  if (dfloat && rr_df_eligible(n_max, m_max)) {
    launch_rr_df(d_tasks, ntask, st, n_max, m_max);
    return;
  }
  const size_t sm = (n_max > 0) ? rr_smem_bytes(n_max, m_max) : (size_t)-1;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (m_max <= RRS_THREADS && sm + 2048 <= (size_t)optin)
    rr_smem_kernel<<<ntask, RRS_THREADS, sm, st>>>(d_tasks);
  else
    rr_kernel<<<ntask, RR_THREADS, 0, st>>>(d_tasks);
}

}  // namespace dgdft
