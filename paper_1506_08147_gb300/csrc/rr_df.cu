// Double-float Rayleigh-Ritz for the FP32 LOBPCG stage (Sec. II.B, operation 4).
//
// The same reduction as the FP64 kernels in dense.cu: equilibrated Cholesky
// of B with its condition check and the LOBPCG fallbacks (drop P, then W,
// then restart), C = L^-1 A L^-T, Householder tridiagonalisation, Sturm-count
// location of the lowest m eigenvalues, inverse iteration with cluster
// re-orthogonalisation, back-transformation and Y = D L^-T Z.  It is carried
// out in double-float arithmetic (dfloat.cuh, about 2^-46 relative), far
// below the ~1e-7 relative error that the FP32 stage's Gram blocks already
// carry, on the FP32 pipes: this part issues about 104 FP32 FMAs per cycle
// and SM against 1.9 FP64 FMAs, and a double-float FMA costs about 13 FP32
// operations.  Scalars (square roots, reciprocal pivots) are formed in FP64
// by one thread.
//
// One CTA (512 threads) per element.  The pencil lives in shared memory with
// an odd leading dimension, so that row and column walks are both free of
// bank conflicts.  Phases that carry a dependency across the whole matrix
// (Cholesky, Householder) are block-synchronous; the triangular solves, the
// back-transformation and the final L^-T solve give every column to one warp
// and need no block barrier.
#include <cfloat>

#include "dfloat.cuh"
#include "internal.h"

namespace dgdft {

namespace {

constexpr int RD_THREADS = 512;
constexpr int RD_WARPS = RD_THREADS / 32;
constexpr int RD_NMAX = 160;             // rows held per lane: RD_NMAX / 32
constexpr int RD_RPL = RD_NMAX / 32;
constexpr int RD_MMAX = 64;              // columns held per warp: RD_MMAX / RD_WARPS
constexpr int RD_CPW = RD_MMAX / RD_WARPS;

struct RdLayout {
  int ld;            // leading dimension of S, Z and the global copies (odd)
  size_t s_dfl;      // S region: the pencil, later the inverse-iteration scratch
  size_t aux_dfl;    // Z region: matvec partials and multisection arrays first
};

__host__ __device__ inline RdLayout rd_layout(int nmax, int m) {
  RdLayout L;
  L.ld = nmax | 1;
  const size_t a = (size_t)nmax * L.ld, b = (size_t)3 * nmax * m;
  L.s_dfl = a > b ? a : b;
  size_t z = (size_t)L.ld * m;
  if (z < (size_t)RD_WARPS * 32) z = (size_t)RD_WARPS * 32;
  if (z < (size_t)nmax + m + RD_THREADS) z = (size_t)nmax + m + RD_THREADS;
  L.aux_dfl = z;
  return L;
}

__host__ __device__ inline size_t rd_smem(int nmax, int m) {
  const RdLayout L = rd_layout(nmax, m);
  return sizeof(dfl) * (L.s_dfl + L.aux_dfl + 5 * (size_t)L.ld + m) + sizeof(double) * 2 * (size_t)m +
         sizeof(int) * (size_t)((m + 1) & ~1);
}

// element (r, c) of the symmetric pencil matrix M: the Gram blocks are formed
// for the upper block triangle, diagonal blocks are averaged with their
// transpose
__device__ __forceinline__ double sym_at(const double* M, int ldm, int r, int c, int bm) {
  const int br = r / bm, bc = c / bm;
  if (br < bc) return M[r + (size_t)c * ldm];
  if (br > bc) return M[c + (size_t)r * ldm];
  return 0.5 * (M[r + (size_t)c * ldm] + M[c + (size_t)r * ldm]);
}

// number of eigenvalues of the tridiagonal (d, e^2) below x, in FP32
__device__ int sturm_below(const float* d, const float* e2, int n, float x) {
  int c = 0;
  float q = 1.0f;
  for (int i = 0; i < n; ++i) {
    q = d[i] - x - ((i > 0) ? __fdividef(e2[i - 1], q) : 0.0f);
    if (fabsf(q) < 1e-30f) q = -1e-30f;
    if (q < 0.0f) ++c;
  }
  return c;
}

__device__ __forceinline__ float hash_unitf(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (float)(h & 0xFFFFFF) * (1.0f / 8388608.0f) - 1.0f;
}

// block-wide sum: the warps' totals go to red, then the warps that read the
// result (warp < nread_warps) add them in one order; returns the sum in
// those warps.  Two barriers.
__device__ __forceinline__ dfl rd_block_sum(dfl v, dfl* red, int nread_warps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = dfl_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  dfl s = dfl_of(0.0f);
  if (warp < nread_warps) {
    s = (lane < RD_WARPS) ? red[lane] : dfl_of(0.0f);
    s = dfl_warp_sum(s);
  }
  return s;
}

// Pivot k of the Cholesky factorisation, by one warp: L_kk = sqrt(S_kk),
// dinv[k] = 1 / L_kk, column k below the diagonal scaled by dinv[k].  A pivot
// that is not positive and finite sets *flag.  Lane 0 tracks the extreme
// pivots.
__device__ __forceinline__ void rd_chol_pivot(dfl* S, int ld, int n, int k, dfl* dinv, int* flag, float* pmin,
                                              float* pmax) {
  const int lane = threadIdx.x & 31;
  dfl* col = S + (size_t)k * ld;
  const dfl p = col[k];
  const bool ok = p.h > 0.0f && isfinite(p.h);
  if (!ok) {
    if (lane == 0) *flag = 1;
    return;
  }
  const dfl inv = dfl_rsqrt(p);
  __syncwarp();
  if (lane == 0) {
    const dfl dk = dfl_mul(p, inv);
    col[k] = dk;
    dinv[k] = inv;
    *pmin = fminf(*pmin, dk.h);
    *pmax = fmaxf(*pmax, dk.h);
  }
  for (int i = k + 1 + lane; i < n; i += 32) col[i] = dfl_mul(col[i], inv);
}

// Householder reflector of column k, by one warp: x = S[k+1.., k],
// alpha = -sign(x_0) |x|, v = (x - alpha e_1) / |x - alpha e_1| written over
// x (zero when x = 0); d[k] = S_kk and e[k] = alpha (x_0 when x = 0).
__device__ __forceinline__ void rd_householder_vector(dfl* S, int ld, int n, int k, dfl* d, dfl* e) {
  const int lane = threadIdx.x & 31;
  dfl* col = S + (size_t)k * ld;
  dfl x[RD_RPL];
  dfl part = dfl_of(0.0f);
#pragma unroll
  for (int r = 0; r < RD_RPL; ++r) {
    const int i = k + 1 + lane + 32 * r;
    x[r] = (i < n) ? col[i] : dfl_of(0.0f);
    part = dfl_fma(x[r], x[r], part);
  }
  const dfl xx = dfl_warp_sum(part);
  const dfl x0 = {__shfl_sync(0xffffffffu, x[0].h, 0), __shfl_sync(0xffffffffu, x[0].l, 0)};
  const dfl dk = col[k];
  __syncwarp();
  if (lane == 0) d[k] = dk;
  if (xx.h > 0.0f) {
    const dfl rx = dfl_rsqrt(xx);
    const dfl nx = dfl_mul(xx, rx);  // |x|
    const dfl alpha = (x0.h >= 0.0f) ? dfl_neg(nx) : nx;
    // |x - alpha e_1|^2 = 2 (|x|^2 + |alpha| |x_0|), no cancellation
    const dfl inv = dfl_rsqrt(dfl_scale2(dfl_fma(nx, dfl_abs(x0), xx), 2.0f));
    if (lane == 0) {
      e[k] = alpha;
      x[0] = dfl_sub(x[0], alpha);
    }
#pragma unroll
    for (int r = 0; r < RD_RPL; ++r) {
      const int i = k + 1 + lane + 32 * r;
      if (i < n) col[i] = dfl_mul(x[r], inv);
    }
  } else {
    if (lane == 0) e[k] = x0;
#pragma unroll
    for (int r = 0; r < RD_RPL; ++r) {
      const int i = k + 1 + lane + 32 * r;
      if (i < n) col[i] = dfl_of(0.0f);
    }
  }
}

// Eigenvectors of the symmetric tridiagonal (d, e) for the m lowest
// eigenvalue estimates lam[] by inverse iteration in double-float; thread q
// owns vector q (column q of Z).  The elimination with partial pivoting
// keeps the rows it finalises (reciprocal pivot and the two entries right of
// it) in scr, interleaved by vector.  Estimates closer than ortol form
// clusters whose shifts are kept apart and whose vectors are orthogonalised
// by modified Gram-Schmidt after every step; isolated vectors take the
// Rayleigh quotient as the shift after the first step.  If any two vectors
// still overlap, the iteration is redone with all m in one cluster.  On
// return the columns are orthonormal and lam[] holds their Rayleigh
// quotients.  Every thread of the block calls.
__device__ void rd_eigvecs(const dfl* d, const dfl* e, int n, int m, double* lam, dfl* Z, int ldz, dfl* scr,
                           int* cstart, double* shift, dfl* dots, double ortol, double gnorm, dfl* red,
                           double* sc, unsigned seed) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double sep = 1e-13 * fmax(gnorm, 1e-300);
  const float tiny = (float)(5.7e-14 * fmax(gnorm, 1e-30));
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
      if (tid < m) {
        const int q = tid;
        dfl* b = Z + (size_t)q * ldz;
        const bool single = cstart[q] == q && (q + 1 >= m || cstart[q + 1] != q);
        if (it == 0)
          for (int i = 0; i < n; ++i) b[i] = dfl_of(hash_unitf(i, q + 7919u * seed));
        dfl lq = dfl_of(shift[q]);
        if (single && it > 0) {
          dfl r0 = dfl_of(0.0f), r1 = dfl_of(0.0f);
          for (int i = 0; i < n; ++i) {
            dfl t = dfl_mul(d[i], b[i]);
            if (i > 0) t = dfl_fma(e[i - 1], b[i - 1], t);
            if (i + 1 < n) t = dfl_fma(e[i], b[i + 1], t);
            if (i & 1) r1 = dfl_fma(b[i], t, r1);
            else r0 = dfl_fma(b[i], t, r0);
          }
          lq = dfl_add(r0, r1);
        }
        // (T - lq I) x = b: elimination with partial pivoting, the current
        // row (c0, c1) at columns (i, i+1) carried in registers
        dfl c0 = dfl_sub(d[0], lq), c1 = (n > 1) ? e[0] : dfl_of(0.0f);
        dfl bi = b[0];
        for (int i = 0; i + 1 < n; ++i) {
          const dfl sub = e[i];
          const dfl n0 = dfl_sub(d[i + 1], lq);
          const dfl n1 = (i + 2 < n) ? e[i + 1] : dfl_of(0.0f);
          const dfl bn = b[i + 1];
          dfl p0, p1, p2, pb;
          if (fabsf(sub.h) > fabsf(c0.h)) {
            const dfl mlt = dfl_mul(c0, dfl_rcp(sub));
            p0 = sub;
            p1 = n0;
            p2 = n1;
            pb = bn;
            c0 = dfl_fnma(mlt, n0, c1);
            c1 = dfl_neg(dfl_mul(mlt, n1));
            bi = dfl_fnma(mlt, bn, bi);
          } else {
            if (fabsf(c0.h) < tiny) c0 = dfl_of(c0.h >= 0.0f ? tiny : -tiny);
            const dfl mlt = dfl_mul(sub, dfl_rcp(c0));
            p0 = c0;
            p1 = c1;
            p2 = dfl_of(0.0f);
            pb = bi;
            c0 = dfl_fnma(mlt, c1, n0);
            c1 = n1;
            bi = dfl_fnma(mlt, bi, bn);
          }
          if (fabsf(p0.h) < tiny) p0 = dfl_of(p0.h >= 0.0f ? tiny : -tiny);
          scr[(size_t)(3 * i) * m + q] = dfl_rcp(p0);
          scr[(size_t)(3 * i + 1) * m + q] = p1;
          scr[(size_t)(3 * i + 2) * m + q] = p2;
          b[i] = pb;
        }
        if (fabsf(c0.h) < tiny) c0 = dfl_of(c0.h >= 0.0f ? tiny : -tiny);
        // back substitution, scaled by the largest entry before the norm
        dfl x1 = dfl_mul(bi, dfl_rcp(c0)), x2 = dfl_of(0.0f);
        b[n - 1] = x1;
        float amax = fabsf(x1.h);
        for (int i = n - 2; i >= 0; --i) {
          dfl s = dfl_fnma(scr[(size_t)(3 * i + 1) * m + q], x1, b[i]);
          s = dfl_fnma(scr[(size_t)(3 * i + 2) * m + q], x2, s);
          const dfl x = dfl_mul(s, scr[(size_t)(3 * i) * m + q]);
          b[i] = x;
          amax = fmaxf(amax, fabsf(x.h));
          x2 = x1;
          x1 = x;
        }
        const dfl sa = dfl_of(amax > 0.0f ? 1.0f / amax : 1.0f);
        dfl n0 = dfl_of(0.0f), n1 = dfl_of(0.0f);
        for (int i = 0; i < n; ++i) {
          const dfl x = dfl_mul(b[i], sa);
          b[i] = x;
          if (i & 1) n1 = dfl_fma(x, x, n1);
          else n0 = dfl_fma(x, x, n0);
        }
        const dfl inv = dfl_of(1.0 / sqrt(dfl_val(dfl_add(n0, n1))));
        for (int i = 0; i < n; ++i) b[i] = dfl_mul(b[i], inv);
      }
      __syncthreads();
      if (!any_cluster) continue;
      for (int j = 0; j < m; ++j) {
        const bool clustered = (cstart[j] != j) || (j + 1 < m && cstart[j + 1] == cstart[j]);
        if (!clustered) continue;  // uniform across the block
        dfl* zj = Z + (size_t)j * ldz;
        dfl part = dfl_of(0.0f);
        for (int i = tid; i < n; i += RD_THREADS) part = dfl_fma(zj[i], zj[i], part);
        const dfl nn = rd_block_sum(part, red, 1);
        if (tid == 0) sc[0] = 1.0 / sqrt(dfl_val(nn));
        __syncthreads();
        const dfl inv = dfl_of(sc[0]);
        for (int i = tid; i < n; i += RD_THREADS) zj[i] = dfl_mul(zj[i], inv);
        __syncthreads();
        int kend = j + 1;
        while (kend < m && cstart[kend] == cstart[j]) ++kend;
        for (int k = j + 1 + warp; k < kend; k += RD_WARPS) {
          const dfl* zk = Z + (size_t)k * ldz;
          dfl s2 = dfl_of(0.0f);
          for (int i = lane; i < n; i += 32) s2 = dfl_fma(zj[i], zk[i], s2);
          s2 = dfl_warp_sum(s2);
          if (lane == 0) dots[k] = s2;
        }
        __syncthreads();
        for (int k = j + 1 + warp; k < kend; k += RD_WARPS) {
          dfl* zk = Z + (size_t)k * ldz;
          const dfl dk = dots[k];
          for (int i = lane; i < n; i += 32) zk[i] = dfl_fnma(dk, zj[i], zk[i]);
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
    for (int t = warp; t < m * REACH; t += RD_WARPS) {
      const int j = t / REACH, k = j + 1 + (t - j * REACH);
      if (k >= m) continue;
      const dfl* zj = Z + (size_t)j * ldz;
      const dfl* zk = Z + (size_t)k * ldz;
      dfl s2 = dfl_of(0.0f);
      for (int i = lane; i < n; i += 32) s2 = dfl_fma(zj[i], zk[i], s2);
      s2 = dfl_warp_sum(s2);
      if (lane == 0 && fabsf(s2.h) > 1e-3f) overlap = 1;
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
  // eigenvalues as Rayleigh quotients z^T T z of the unit vectors
  for (int j = warp; j < m; j += RD_WARPS) {
    const dfl* zj = Z + (size_t)j * ldz;
    dfl s5 = dfl_of(0.0f);
    for (int i = lane; i < n; i += 32) {
      dfl t = dfl_mul(d[i], zj[i]);
      if (i > 0) t = dfl_fma(e[i - 1], zj[i - 1], t);
      if (i + 1 < n) t = dfl_fma(e[i], zj[i + 1], t);
      s5 = dfl_fma(zj[i], t, s5);
    }
    s5 = dfl_warp_sum(s5);
    if (lane == 0) lam[j] = dfl_val(s5);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RD_THREADS, 1) rr_df_kernel(const RRTask* __restrict__ tasks, int nmax_all,
                                                              int mmax_all) {
  const RRTask T = tasks[blockIdx.x];
  if (T.state && !T.state[ST_ACTIVE]) return;
  if (T.state && (T.state[ST_ERROR] & ERR_TIMEOUT)) {
    // a wait in this iteration's Gram launch ran out: its products are stale
    if (threadIdx.x == 0) T.state[ST_ACTIVE] = 0;
    return;
  }
  const RdLayout Lay = rd_layout(nmax_all, mmax_all);
  const int ld = Lay.ld;
  extern __shared__ __align__(16) unsigned char rd_raw[];
  dfl* S = reinterpret_cast<dfl*>(rd_raw);
  dfl* AUX = S + Lay.s_dfl;
  dfl* Z = AUX;
  dfl* dd = AUX + Lay.aux_dfl;
  dfl* ee = dd + ld;
  dfl* scal = ee + ld;
  dfl* dinv = scal + ld;
  dfl* pv = dinv + ld;
  dfl* dots = pv + ld;
  double* lam = reinterpret_cast<double*>(dots + mmax_all);
  double* shift = lam + mmax_all;
  int* cstart = reinterpret_cast<int*>(shift + mmax_all);
  __shared__ dfl red[RD_WARPS];
  __shared__ float redf[3 * RD_WARPS];
  __shared__ double sc[4];
  __shared__ int sflag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int m = T.m;
  int n = (T.mode == RR_FIXED) ? T.n_fixed
          : (T.mode == RR_INITIAL) ? m
          : (T.state[ST_HAS_P] ? 3 * m : 2 * m);
  const int bm = (T.mode == RR_FIXED) ? n : m;
  const int n_out = (T.mode == RR_LOBPCG) ? 3 * m : n;
  // global copies in the task's own work buffer (sized for its largest
  // pencil, n_out x n_out): L, and the reflectors while S is scratch
  const int ldw = n_out;
  dfl* WL = reinterpret_cast<dfl*>(T.work);
  dfl* WH = WL + (size_t)ldw * ldw;
  bool dropped = false;

  for (;;) {
    // 1. equilibrated B = D B D (lower triangle), D = diag(B)^-1/2
    if (tid == 0) sflag = 0;
    __syncthreads();
    for (int i = tid; i < n; i += RD_THREADS) {
      const double bii = T.B[i + (size_t)i * T.ld];
      if (!(bii > 0.0) || !isfinite(bii)) {
        sflag = 1;
        scal[i] = dfl_of(0.0f);
      } else {
        scal[i] = dfl_of(1.0 / sqrt(bii));
      }
    }
    __syncthreads();
    for (int c = warp; c < n; c += RD_WARPS)
      for (int r = c + lane; r < n; r += 32)
        S[r + (size_t)c * ld] = dfl_mul(dfl_mul(dfl_of(sym_at(T.B, T.ld, r, c, bm)), scal[r]), scal[c]);
    __syncthreads();
    // Cholesky B = L L^T, right-looking on the lower triangle.  Warp 0
    // updates column k+1 first and finishes it (pivot, scaling) while the
    // other warps update the rest, so a step needs one barrier.
    float pmin = FLT_MAX, pmax = 0.0f;  // thread 0's
    if (warp == 0) rd_chol_pivot(S, ld, n, 0, dinv, &sflag, &pmin, &pmax);
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
      if (sflag) break;
      const dfl* lk = S + (size_t)k * ld;
      if (warp == 0) {
        const int j = k + 1;
        const dfl ljk = lk[j];
        dfl* col = S + (size_t)j * ld;
        for (int i = j + lane; i < n; i += 32) col[i] = dfl_fnma(lk[i], ljk, col[i]);
        __syncwarp();
        rd_chol_pivot(S, ld, n, j, dinv, &sflag, &pmin, &pmax);
      } else {
        for (int j = k + 1 + warp; j < n; j += RD_WARPS - 1) {
          const dfl ljk = lk[j];
          dfl* col = S + (size_t)j * ld;
          for (int i = j + lane; i < n; i += 32) col[i] = dfl_fnma(lk[i], ljk, col[i]);
        }
      }
      __syncthreads();
    }
    const bool last_resort = T.mode == RR_LOBPCG && n == m;
    const double cond_lim = last_resort ? (T.restart_max > 0 ? 1e6 : 1e300) : T.cond_max;
    if (tid == 0) {
      const double ratio = (double)pmax / (double)pmin;
      sc[1] = (!sflag && ratio * ratio > cond_lim) ? 1.0 : 0.0;
    }
    // read before the barrier: thread 0 updates the count after it
    const bool can_restart =
        T.mode == RR_LOBPCG && T.restart_max > 0 && T.state && T.state[ST_NRESTART] < T.restart_max;
    __syncthreads();
    const bool fail = sflag != 0 || sc[1] != 0.0;
    __syncthreads();
    if (fail) {
      if (T.mode == RR_LOBPCG && n == 3 * m) {
        n = 2 * m;
        dropped = true;
        continue;
      }
      if (T.mode == RR_LOBPCG && n == 2 * m) {
        // [X W] is numerically dependent too: Rayleigh-Ritz on X alone, a
        // rotation of the current block; the next iteration brings a new W
        n = m;
        dropped = true;
        continue;
      }
      if (can_restart) {
        // no usable pencil, not even X alone: keep X (Y = [I; 0]) and let
        // the restart step perturb it and drop P (Ritz values unchanged)
        const int nr = 3 * m;
        for (int idx = tid; idx < nr * m; idx += RD_THREADS) {
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
    // L to global memory (its reciprocal diagonal is in dinv)
    for (int c = warp; c < n; c += RD_WARPS)
      for (int r = c + lane; r < n; r += 32) WL[r + (size_t)c * ldw] = S[r + (size_t)c * ld];
    __syncthreads();
    // 2. C = L^-1 (D A D) L^-T: A in full (lower triangle read, mirrored),
    // then S <- L^-1 S, S <- S^T, S <- L^-1 S; warp w owns columns w (mod 16)
    for (int c = warp; c < n; c += RD_WARPS)
      for (int r = c + lane; r < n; r += 32) {
        const dfl a = dfl_mul(dfl_mul(dfl_of(sym_at(T.A, T.ld, r, c, bm)), scal[r]), scal[c]);
        S[r + (size_t)c * ld] = a;
        S[c + (size_t)r * ld] = a;
      }
    __syncthreads();
    // each pass solves L Y = S column by column, leaving row k unscaled
    // (S[k, c] L_kk = Y[k, c]); the scaling by 1/L_kk is folded into the
    // transpose after pass 0 and the symmetrisation after pass 1
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = 0; k < n; ++k) {
        const int rows = (n - k - 1 + 31) >> 5;
        dfl lk[RD_RPL];
#pragma unroll
        for (int r = 0; r < RD_RPL; ++r) {
          const int i = k + 1 + lane + 32 * r;
          lk[r] = (r < rows && i < n) ? WL[i + (size_t)k * ldw] : dfl_of(0.0f);
        }
        const dfl dk = dinv[k];
#pragma unroll 2
        for (int c = warp; c < n; c += RD_WARPS) {
          dfl* col = S + (size_t)c * ld;
          const dfl y = dfl_mul(col[k], dk);
#pragma unroll
          for (int r = 0; r < RD_RPL; ++r) {
            const int i = k + 1 + lane + 32 * r;
            if (r < rows && i < n) col[i] = dfl_fnma(lk[r], y, col[i]);
          }
        }
        __syncwarp();
      }
      __syncthreads();
      if (pass == 0) {
        // S <- (D^-1 S)^T with D = diag(L)
        for (int c = warp; c < n; c += RD_WARPS)
          for (int r = lane; r <= c; r += 32) {
            const dfl a = dfl_mul(S[r + (size_t)c * ld], dinv[r]);
            const dfl b = dfl_mul(S[c + (size_t)r * ld], dinv[c]);
            S[r + (size_t)c * ld] = b;
            S[c + (size_t)r * ld] = a;
          }
        __syncthreads();
      }
    }
    // C = D^-1 S; its lower triangle takes the mean of C and C^T
    for (int c = warp; c < n; c += RD_WARPS)
      for (int r = c + lane; r < n; r += 32) {
        const dfl a = dfl_mul(S[r + (size_t)c * ld], dinv[r]);
        const dfl b = dfl_mul(S[c + (size_t)r * ld], dinv[c]);
        S[r + (size_t)c * ld] = (r == c) ? a : dfl_scale2(dfl_add(a, b), 0.5f);
      }
    __syncthreads();
    // 3. Householder tridiagonalisation on the lower triangle; reflector k
    // (unit vector v, H = I - 2 v v^T) kept in S[k+1.., k].  A step: p = C v
    // by 32-row groups x column parts, with the parts' shares of v^T p;
    // p' = 2 (p - (v^T p) v); C -= v p'^T + p' v^T, where warp 0 updates
    // column k+1 first and forms the next reflector from it.
    if (n >= 3 && warp == 0) rd_householder_vector(S, ld, n, 0, dd, ee);
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
      const int nk = n - k - 1;
      const dfl* vk = S + (size_t)k * ld;
      const int G = (nk + 31) >> 5;
      const int P = RD_WARPS / G;
      if (warp < G * P) {
        const int g = warp % G, pp = warp / G;
        const int chunk = (nk + P - 1) / P;
        const int i = k + 1 + 32 * g + lane;
        const int j0 = k + 1 + pp * chunk;
        const int j1 = min(n, j0 + chunk);
        dfl s0 = dfl_of(0.0f), s1 = dfl_of(0.0f), kp = dfl_of(0.0f);
        if (i < n) {
          int j = j0;
          for (; j + 1 < j1; j += 2) {
            const dfl a0 = (j <= i) ? S[i + (size_t)j * ld] : S[j + (size_t)i * ld];
            const dfl a1 = (j + 1 <= i) ? S[i + (size_t)(j + 1) * ld] : S[j + 1 + (size_t)i * ld];
            s0 = dfl_fma(a0, vk[j], s0);
            s1 = dfl_fma(a1, vk[j + 1], s1);
          }
          if (j < j1) {
            const dfl a0 = (j <= i) ? S[i + (size_t)j * ld] : S[j + (size_t)i * ld];
            s0 = dfl_fma(a0, vk[j], s0);
          }
          s0 = dfl_add(s0, s1);
          kp = dfl_mul(vk[i], s0);
        }
        AUX[warp * 32 + lane] = s0;
        kp = dfl_warp_sum(kp);
        if (lane == 0) red[warp] = kp;
      }
      __syncthreads();
      if (warp < G) {
        dfl K = (lane < G * P) ? red[lane] : dfl_of(0.0f);
        K = dfl_warp_sum(K);
        const int i = k + 1 + tid;
        if (i < n) {
          dfl p = AUX[warp * 32 + lane];
          for (int q = 1; q < P; ++q) p = dfl_add(p, AUX[(warp + q * G) * 32 + lane]);
          pv[i] = dfl_scale2(dfl_fnma(K, vk[i], p), 2.0f);
        }
      }
      __syncthreads();
      if (warp == 0) {
        const int j = k + 1;
        const dfl vj = vk[j], pj = pv[j];
        dfl* col = S + (size_t)j * ld;
        for (int i = j + lane; i < n; i += 32) col[i] = dfl_fnma(vk[i], pj, dfl_fnma(pv[i], vj, col[i]));
        __syncwarp();
        if (k + 3 < n) rd_householder_vector(S, ld, n, j, dd, ee);
      } else {
        for (int j = k + 1 + warp; j < n; j += RD_WARPS - 1) {
          const dfl vj = vk[j], pj = pv[j];
          dfl* col = S + (size_t)j * ld;
          for (int i = j + lane; i < n; i += 32) col[i] = dfl_fnma(vk[i], pj, dfl_fnma(pv[i], vj, col[i]));
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        dd[n - 2] = S[n - 2 + (size_t)(n - 2) * ld];
        ee[n - 2] = S[n - 1 + (size_t)(n - 2) * ld];
      }
      dd[n - 1] = S[n - 1 + (size_t)(n - 1) * ld];
      ee[n - 1] = dfl_of(0.0f);
    }
    // the reflectors to global memory: S becomes inverse-iteration scratch
    for (int c = warp; c + 2 < n; c += RD_WARPS)
      for (int r = c + 1 + lane; r < n; r += 32) WH[r + (size_t)c * ldw] = S[r + (size_t)c * ld];
    __syncthreads();
    // 4. eigenvalue shifts by FP32 multisection of the Sturm count: tper
    // threads per eigenvalue split its bracket into tper + 1 parts a round
    float* d32 = reinterpret_cast<float*>(AUX);
    float* e2 = d32 + n;
    float* lo_s = e2 + n;
    float* hi_s = lo_s + m;
    float* xs = hi_s + m;
    int* cnt = reinterpret_cast<int*>(xs + RD_THREADS);
    float glo = FLT_MAX, ghi = -FLT_MAX, gno = 0.0f;
    for (int i = tid; i < n; i += RD_THREADS) {
      const float di = dd[i].h + dd[i].l;
      const float ei = ee[i].h;
      const float r = (i > 0 ? fabsf(ee[i - 1].h) : 0.0f) + (i < n - 1 ? fabsf(ei) : 0.0f);
      d32[i] = di;
      e2[i] = ei * ei;
      glo = fminf(glo, di - r);
      ghi = fmaxf(ghi, di + r);
      gno = fmaxf(gno, fabsf(di) + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
      ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
      gno = fmaxf(gno, __shfl_xor_sync(0xffffffffu, gno, o));
    }
    if (lane == 0) {
      redf[warp] = glo;
      redf[RD_WARPS + warp] = ghi;
      redf[2 * RD_WARPS + warp] = gno;
    }
    __syncthreads();
    glo = redf[0];
    ghi = redf[RD_WARPS];
    gno = redf[2 * RD_WARPS];
    for (int w = 1; w < RD_WARPS; ++w) {
      glo = fminf(glo, redf[w]);
      ghi = fmaxf(ghi, redf[RD_WARPS + w]);
      gno = fmaxf(gno, redf[2 * RD_WARPS + w]);
    }
    const double gnorm = (double)fmaxf(gno, 1e-30f);
    const int tper = RD_THREADS / m;
    const int jv = tid / tper, sv = tid - jv * tper;
    {
      const float pad = 1e-6f * (float)gnorm;
      for (int j = tid; j < m; j += RD_THREADS) {
        lo_s[j] = glo - pad;
        hi_s[j] = ghi + pad;
      }
      __syncthreads();
      const int rounds = (int)ceilf(40.0f / log2f((float)(tper + 1)));
      for (int rd = 0; rd < rounds; ++rd) {
        if (jv < m) {
          const float lo = lo_s[jv], hi = hi_s[jv];
          const float x = lo + (hi - lo) * ((float)(sv + 1) / (float)(tper + 1));
          xs[tid] = x;
          cnt[tid] = (x > lo && x < hi) ? sturm_below(d32, e2, n, x) : -1;
        }
        __syncthreads();
        if (jv < m && sv == 0) {
          float lo = lo_s[jv], hi = hi_s[jv];
          for (int q = 0; q < tper; ++q) {
            const int c = cnt[tid + q];
            if (c < 0) break;
            if (c > jv) {
              hi = xs[tid + q];
              break;
            }
            lo = xs[tid + q];
          }
          lo_s[jv] = lo;
          hi_s[jv] = hi;
        }
        __syncthreads();
      }
      for (int j = tid; j < m; j += RD_THREADS) lam[j] = 0.5 * ((double)lo_s[j] + (double)hi_s[j]);
      __syncthreads();
    }
    // 5. eigenvectors by inverse iteration (Z aliases the multisection arrays,
    // which are dead now; S is the elimination scratch)
    rd_eigvecs(dd, ee, n, m, lam, Z, ld, S, cstart, shift, dots, 1e-5 * gnorm, gnorm, red, sc, blockIdx.x);
    for (int c = warp; c + 2 < n; c += RD_WARPS)
      for (int r = c + 1 + lane; r < n; r += 32) S[r + (size_t)c * ld] = WH[r + (size_t)c * ldw];
    __syncthreads();
    // 6. back-transformation x = H_0 ... H_{n-3} z, warp w owning columns
    // w (mod 16) of Z in registers (rows lane + 32 r)
    dfl z[RD_CPW][RD_RPL];
    const int ncw = (m - warp + RD_WARPS - 1) / RD_WARPS;  // columns this warp owns
#pragma unroll
    for (int cc = 0; cc < RD_CPW; ++cc) {
      const int c = warp + RD_WARPS * cc;
#pragma unroll
      for (int r = 0; r < RD_RPL; ++r) {
        const int i = lane + 32 * r;
        z[cc][r] = (c < m && i < n) ? Z[i + (size_t)c * ld] : dfl_of(0.0f);
      }
    }
    for (int k = n - 3; k >= 0; --k) {
      const dfl* vk = S + (size_t)k * ld;
      const int rlo = (k + 1) >> 5;  // row chunks below rlo are untouched by H_k
      dfl v[RD_RPL];
#pragma unroll
      for (int r = 0; r < RD_RPL; ++r) {
        const int i = lane + 32 * r;
        v[r] = (r >= rlo && i > k && i < n) ? vk[i] : dfl_of(0.0f);
      }
      dfl s[RD_CPW];
#pragma unroll
      for (int cc = 0; cc < RD_CPW; ++cc) {
        dfl a = dfl_of(0.0f);
        if (cc < ncw)
#pragma unroll
          for (int r = 0; r < RD_RPL; ++r)
            if (r >= rlo) a = dfl_fma(v[r], z[cc][r], a);
        s[cc] = a;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int cc = 0; cc < RD_CPW; ++cc)
          if (cc < ncw) {
            const dfl w = {__shfl_down_sync(0xffffffffu, s[cc].h, o), __shfl_down_sync(0xffffffffu, s[cc].l, o)};
            s[cc] = dfl_add(s[cc], w);
          }
#pragma unroll
      for (int cc = 0; cc < RD_CPW; ++cc)
        if (cc < ncw) {
          const dfl t = dfl_scale2(
              dfl{__shfl_sync(0xffffffffu, s[cc].h, 0), __shfl_sync(0xffffffffu, s[cc].l, 0)}, 2.0f);
#pragma unroll
          for (int r = 0; r < RD_RPL; ++r)
            if (r >= rlo) z[cc][r] = dfl_fnma(t, v[r], z[cc][r]);
        }
    }
    __syncthreads();
    // 7. Y = D L^-T x: L back into S, then backward substitution per column
    for (int c = warp; c < n; c += RD_WARPS)
      for (int r = c + lane; r < n; r += 32) S[r + (size_t)c * ld] = WL[r + (size_t)c * ldw];
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
      const dfl di = dinv[i];
      const int src = i & 31, ri = i >> 5;
      dfl li[RD_RPL];
#pragma unroll
      for (int r = 0; r < RD_RPL; ++r) {
        const int k = lane + 32 * r;
        li[r] = (k < i) ? S[i + (size_t)k * ld] : dfl_of(0.0f);
      }
#pragma unroll
      for (int cc = 0; cc < RD_CPW; ++cc) {
        if (cc >= ncw) continue;
        dfl zi = z[cc][0];
#pragma unroll
        for (int r = 1; r < RD_RPL; ++r)
          if (r == ri) zi = z[cc][r];
        zi = dfl{__shfl_sync(0xffffffffu, zi.h, src), __shfl_sync(0xffffffffu, zi.l, src)};
        const dfl yi = dfl_mul(zi, di);
#pragma unroll
        for (int r = 0; r < RD_RPL; ++r) {
          if (r == ri && lane == src) z[cc][r] = yi;
          else if (r <= ri) z[cc][r] = dfl_fnma(li[r], yi, z[cc][r]);  // rows k < i only
        }
      }
    }
#pragma unroll
    for (int cc = 0; cc < RD_CPW; ++cc) {
      const int c = warp + RD_WARPS * cc;
      if (c >= m) continue;
#pragma unroll
      for (int r = 0; r < RD_RPL; ++r) {
        const int row = lane + 32 * r;
        if (row >= n_out) continue;
        const double y = (row < n) ? dfl_val(dfl_mul(z[cc][r], scal[row])) : 0.0;
        T.Y[row + (size_t)c * T.ldy] = y;
        if (T.Yf) T.Yf[row + (size_t)c * T.ldy] = (float)y;
      }
    }
    for (int c = tid; c < m; c += RD_THREADS) T.theta[c] = lam[c];
    if (tid == 0 && dropped && T.state) T.state[ST_FALLBACK] += 1;
    return;
  }
}

}  // namespace

bool rr_df_eligible(int n_max, int m_max) {
  if (n_max < 1 || m_max < 1 || n_max > RD_NMAX || m_max > RD_MMAX || m_max > n_max) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  // static shared memory of the kernel: red, redf, sc, flags
  return rd_smem(n_max, m_max) + 1024 <= (size_t)optin;
}

void init_rr_df_kernel() { opt_in_dynamic_smem((const void*)rr_df_kernel); }

void launch_rr_df(const RRTask* d_tasks, int ntask, cudaStream_t st, int n_max, int m_max) {
  if (ntask <= 0) return;
  rr_df_kernel<<<ntask, RD_THREADS, rd_smem(n_max, m_max), st>>>(d_tasks, n_max, m_max);
}

}  // namespace dgdft
