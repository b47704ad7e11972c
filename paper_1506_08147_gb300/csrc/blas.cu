// Tall-skinny block operations of LOBPCG (Sec. II.B, operations 2 and 3).
//
// Each iteration forms 12 Gram products Phi^T Psi (the 6 + 6 distinct blocks
// of S^T H S and S^T S, S = [X W P]) and 7 block updates Phi C with small C.
// The paper splits rows over a processor column group and sums the J x J
// partial products with MPI_Allreduce; here the row split is over CTAs
// (split-K) and the partial products are summed on the device in a fixed
// order, so results do not depend on scheduling.
//
// These are the SIMT kernels (FP64 for the plain solver, FP32 accumulation
// within a chunk for the mixed form); partial sums are always FP64.
#include "internal.h"

namespace dgdft {

namespace {

constexpr int TILE = 64;   // output tile edge
constexpr int KS = 32;     // rows staged per shared-memory step (Gram)
constexpr int KU = 16;     // inner dimension staged per step (update)
constexpr double SHIFT_RES = 5e-2;  // residual below which the FP32 shift follows the Ritz values

template <class real>
__device__ __forceinline__ int ld_of(const ElemDev<real>& e, const BRef<real>& r, int ld_in, int rows) {
  return r.ptr ? (ld_in > 0 ? ld_in : rows) : e.ng;
}

// grid: (nchunk, npairs * tiles_a * tiles_b, nel); block 256 = 16 x 16.
template <class real>
__global__ void __launch_bounds__(256) gram_kernel(const ElemDev<real>* __restrict__ elems,
                                                   GramJob<real> job, double* __restrict__ partial,
                                                   size_t pstride, int kchunk, int tiles_a,
                                                   int tiles_b) {
  __shared__ real As[KS][TILE + 4];
  __shared__ real Bs[KS][TILE + 4];
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int ntile = tiles_a * tiles_b;
  const int pair = blockIdx.y / ntile;
  const int t = blockIdx.y - pair * ntile;
  const int ta = t / tiles_b, tb = t - ta * tiles_b;
  if (job.needs_p[pair] && !e.state[ST_HAS_P]) return;
  const int ca = job.ncols_a > 0 ? job.ncols_a : e.m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const int a0 = ta * TILE, b0 = tb * TILE;
  if (a0 >= ca || b0 >= cb) return;
  const real* A = resolve(e, job.a[pair]);
  const real* B = resolve(e, job.b[pair]);
  const int lda = ld_of(e, job.a[pair], job.ld_in, rows);
  const int ldb = ld_of(e, job.b[pair], job.ld_in, rows);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k_beg = blockIdx.x * kchunk;
  const int k_end = min(rows, k_beg + kchunk);
  real acc[4][4];
  // FP32: each KS-row step is summed in FP32 and folded into a compensated
  // (hi, lo) pair, so rounding does not grow with the chunk length (the
  // Gram entries carry residual information ~1e-6 of their size)
  real chi[4][4], clo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = chi[i][j] = clo[i][j] = 0;
  for (int k0 = k_beg; k0 < k_end; k0 += KS) {
    for (int i = threadIdx.x; i < KS * TILE; i += blockDim.x) {
      const int c = i / KS, r = i - c * KS;
      const int k = k0 + r;
      const bool kin = k < k_end;
      As[r][c] = (kin && a0 + c < ca) ? A[(size_t)(a0 + c) * lda + k] : (real)0;
      Bs[r][c] = (kin && b0 + c < cb) ? B[(size_t)(b0 + c) * ldb + k] : (real)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < KS; ++r) {
      real av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[r][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[r][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
    if constexpr (sizeof(real) == sizeof(float)) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // Knuth's two-sum of chi + acc: exact error term into clo
          const real sum = chi[i][j] + acc[i][j];
          const real bp = sum - chi[i][j];
          clo[i][j] += (chi[i][j] - (sum - bp)) + (acc[i][j] - bp);
          chi[i][j] = sum;
          acc[i][j] = 0;
        }
    }
  }
  double* out = partial + blockIdx.z * pstride +
                ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * (TILE * TILE);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      out[(ty * 4 + i) * TILE + tx * 4 + j] = (double)acc[i][j] + (double)chi[i][j] + (double)clo[i][j];
}

// FP32 Gram products for blocks of at most 48 columns (the LOBPCG pencil at
// m <= 48): one 48 x 48 output tile per CTA of 144 threads (4 x 4 outputs
// each), the pairs of one row chunk adjacent in the grid so the blocks they
// share come from L2.  Operands are staged column-major (rows contiguous)
// by double-buffered cp.async; each thread reads 4 rows of a column as one
// float4, with the 16-byte chunks of a column XOR-swizzled by column group
// so the twelve column groups of a warp hit distinct banks.  Accumulation
// as in gram_kernel: FP32 per 32-row stage, folded into a two-sum
// compensated pair.  Partials use gram_kernel's 64 x 64 layout.
// grid: (npairs, nchunk, nel); block 144.
constexpr int G48 = 48;
constexpr int GK = 32;  // rows per stage

__device__ __forceinline__ int g48_off(int c, int r) {
  return c * GK + ((((r >> 2) ^ ((c >> 2) & 7)) << 2) | (r & 3));
}

__global__ void __launch_bounds__(144) gram48_kernel(const ElemDev<float>* __restrict__ elems,
                                                      GramJob<float> job, double* __restrict__ partial,
                                                      size_t pstride, int kchunk) {
  __shared__ __align__(16) float As[2][G48 * GK];
  __shared__ __align__(16) float Bs[2][G48 * GK];
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int pair = blockIdx.x;
  if (job.needs_p[pair] && !e.state[ST_HAS_P]) return;
  const int ca = job.ncols_a > 0 ? job.ncols_a : e.m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const float* A = resolve(e, job.a[pair]);
  const float* B = resolve(e, job.b[pair]);
  const int lda = ld_of(e, job.a[pair], job.ld_in, rows);
  const int ldb = ld_of(e, job.b[pair], job.ld_in, rows);
  const int tx = threadIdx.x % 12, ty = threadIdx.x / 12;
  const int k_beg = blockIdx.y * kchunk;
  const int k_end = min(rows, k_beg + kchunk);
  // 16-byte copies need 16-byte aligned column starts
  const bool vec = ((lda | ldb | k_beg) & 3) == 0 && ((((uintptr_t)A) | ((uintptr_t)B)) & 15) == 0;
  auto load_stage = [&](int buf, int k0) {
    for (int t = threadIdx.x; t < 2 * G48 * (GK / 4); t += blockDim.x) {
      const int op = t / (G48 * (GK / 4));
      const int rem = t - op * (G48 * (GK / 4));
      const int c = rem / (GK / 4), q = rem - c * (GK / 4);
      const float* src = op ? B : A;
      const int ld = op ? ldb : lda;
      const int cc = op ? cb : ca;
      float* dst = (op ? Bs[buf] : As[buf]) + g48_off(c, 4 * q);
      const int k = k0 + 4 * q;
      const int nv = (c < cc) ? max(0, min(4, k_end - k)) : 0;
      const float* g = nv ? src + (size_t)c * ld + k : src;
      if (vec) {
        cp_async16(dst, g, 4 * nv);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) cp_async4(dst + u, u < nv ? g + u : src, u < nv ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  float acc[4][4], chi[4][4], clo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = chi[i][j] = clo[i][j] = 0.f;
  const int nst = (k_end > k_beg) ? (k_end - k_beg + GK - 1) / GK : 0;
  if (nst > 0) load_stage(0, k_beg);
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) {
      load_stage((st + 1) & 1, k_beg + (st + 1) * GK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* as = As[st & 1];
    const float* bs = Bs[st & 1];
#pragma unroll 2
    for (int r = 0; r < GK; r += 4) {
      float4 a4[4], b4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a4[i] = *reinterpret_cast<const float4*>(as + g48_off(ty * 4 + i, r));
#pragma unroll
      for (int j = 0; j < 4; ++j) b4[j] = *reinterpret_cast<const float4*>(bs + g48_off(tx * 4 + j, r));
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float t = acc[i][j];
          t = fmaf(a4[i].x, b4[j].x, t);
          t = fmaf(a4[i].y, b4[j].y, t);
          t = fmaf(a4[i].z, b4[j].z, t);
          t = fmaf(a4[i].w, b4[j].w, t);
          acc[i][j] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float sum = chi[i][j] + acc[i][j];
        const float bp = sum - chi[i][j];
        clo[i][j] += (chi[i][j] - (sum - bp)) + (acc[i][j] - bp);
        chi[i][j] = sum;
        acc[i][j] = 0.f;
      }
  }
  double* out = partial + blockIdx.z * pstride + ((size_t)blockIdx.y * gridDim.x + pair) * (TILE * TILE);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * TILE + tx * 4 + j] = (double)chi[i][j] + (double)clo[i][j];
}

// FP64 Gram products for blocks of at most 48 columns (the FP64 stage at
// m <= 48): the layout of gram48_kernel with 16-row stages of doubles, each
// thread reading 2 rows of a column as one 16-byte double2 (chunks of a
// column swizzled by column group as there).  FP64 accumulation; the FP64
// pipe bounds it, and 48-wide tiles avoid the 64-wide tiles' idle lanes.
// grid: (npairs, nchunk, nel); block 144.
constexpr int GKD = 16;  // rows per stage (doubles)

__device__ __forceinline__ int g48d_off(int c, int r) {
  return c * GKD + ((((r >> 1) ^ ((c >> 2) & 7)) << 1) | (r & 1));
}

__global__ void __launch_bounds__(144) gram48d_kernel(const ElemDev<double>* __restrict__ elems,
                                                       GramJob<double> job, double* __restrict__ partial,
                                                       size_t pstride, int kchunk) {
  __shared__ __align__(16) double As[2][G48 * GKD];
  __shared__ __align__(16) double Bs[2][G48 * GKD];
  const ElemDev<double>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int pair = blockIdx.x;
  if (job.needs_p[pair] && !e.state[ST_HAS_P]) return;
  const int ca = job.ncols_a > 0 ? job.ncols_a : e.m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const double* A = resolve(e, job.a[pair]);
  const double* B = resolve(e, job.b[pair]);
  const int lda = ld_of(e, job.a[pair], job.ld_in, rows);
  const int ldb = ld_of(e, job.b[pair], job.ld_in, rows);
  const int tx = threadIdx.x % 12, ty = threadIdx.x / 12;
  const int k_beg = blockIdx.y * kchunk;
  const int k_end = min(rows, k_beg + kchunk);
  const bool vec = ((lda | ldb | k_beg) & 1) == 0 && ((((uintptr_t)A) | ((uintptr_t)B)) & 15) == 0;
  auto load_stage = [&](int buf, int k0) {
    for (int t = threadIdx.x; t < 2 * G48 * (GKD / 2); t += blockDim.x) {
      const int op = t / (G48 * (GKD / 2));
      const int rem = t - op * (G48 * (GKD / 2));
      const int c = rem / (GKD / 2), q = rem - c * (GKD / 2);
      const double* src = op ? B : A;
      const int ld = op ? ldb : lda;
      const int cc = op ? cb : ca;
      double* dst = (op ? Bs[buf] : As[buf]) + g48d_off(c, 2 * q);
      const int k = k0 + 2 * q;
      const int nv = (c < cc) ? max(0, min(2, k_end - k)) : 0;
      const double* g = nv ? src + (size_t)c * ld + k : src;
      if (vec) {
        cp_async16(dst, g, 8 * nv);
      } else {
        // 8-byte pieces: two 4-byte copies each
        const float* gf = reinterpret_cast<const float*>(g);
        const float* sf = reinterpret_cast<const float*>(src);
        float* df = reinterpret_cast<float*>(dst);
#pragma unroll
        for (int u = 0; u < 4; ++u) cp_async4(df + u, u < 2 * nv ? gf + u : sf, u < 2 * nv ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int nst = (k_end > k_beg) ? (k_end - k_beg + GKD - 1) / GKD : 0;
  if (nst > 0) load_stage(0, k_beg);
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) {
      load_stage((st + 1) & 1, k_beg + (st + 1) * GKD);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const double* as = As[st & 1];
    const double* bs = Bs[st & 1];
#pragma unroll 2
    for (int r = 0; r < GKD; r += 2) {
      double2 a2[4], b2[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a2[i] = *reinterpret_cast<const double2*>(as + g48d_off(ty * 4 + i, r));
#pragma unroll
      for (int j = 0; j < 4; ++j) b2[j] = *reinterpret_cast<const double2*>(bs + g48d_off(tx * 4 + j, r));
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a2[i].y, b2[j].y, fma(a2[i].x, b2[j].x, acc[i][j]));
    }
    __syncthreads();
  }
  double* out = partial + blockIdx.z * pstride + ((size_t)blockIdx.y * gridDim.x + pair) * (TILE * TILE);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * TILE + tx * 4 + j] = acc[i][j];
}

// FP64 Gram products in double-float arithmetic (the FP64 stage at m <= 48).
// GB300 runs FP64 at 1/64 of the FP32 rate, and gram48d_kernel is bound by
// it.  Here each staged FP64 value x is split once into FP32 parts
// x = xh + xl (|xl| <= 2^-24 |xh|, the pair carries ~2^-48 of x); a product
// is formed as xh*yh exactly (its rounding error recovered by an FMA) plus
// the cross terms xh*yl + xl*yh, and accumulated into a (hi, lo) FP32 pair
// by a two-sum per product: ~2^-44 relative, at FP32-pipe rates.  The FP64
// stage only needs its pencil far more accurately than the FP32 stage's,
// not to FP64 rounding.  Layout and staging as gram48d_kernel (FP64 blocks
// staged by cp.async), then a conversion pass writes the parts row-major
// ([row][column], 48 floats a row) so a thread reads its four columns as
// one float4.  grid: (npairs, nchunk, nel); block 144.
__global__ void __launch_bounds__(144) gram48df_kernel(const ElemDev<double>* __restrict__ elems,
                                                        GramJob<double> job, double* __restrict__ partial,
                                                        size_t pstride, int kchunk) {
  __shared__ __align__(16) double As[2][G48 * GKD];
  __shared__ __align__(16) double Bs[2][G48 * GKD];
  __shared__ __align__(16) float Ah[GKD][G48], Al[GKD][G48], Bh[GKD][G48], Bl[GKD][G48];
  const ElemDev<double>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int pair = blockIdx.x;
  if (job.needs_p[pair] && !e.state[ST_HAS_P]) return;
  const int ca = job.ncols_a > 0 ? job.ncols_a : e.m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const double* A = resolve(e, job.a[pair]);
  const double* B = resolve(e, job.b[pair]);
  const int lda = ld_of(e, job.a[pair], job.ld_in, rows);
  const int ldb = ld_of(e, job.b[pair], job.ld_in, rows);
  const int tx = threadIdx.x % 12, ty = threadIdx.x / 12;
  const int k_beg = blockIdx.y * kchunk;
  const int k_end = min(rows, k_beg + kchunk);
  const bool vec = ((lda | ldb | k_beg) & 1) == 0 && ((((uintptr_t)A) | ((uintptr_t)B)) & 15) == 0;
  auto load_stage = [&](int buf, int k0) {
    for (int t = threadIdx.x; t < 2 * G48 * (GKD / 2); t += blockDim.x) {
      const int op = t / (G48 * (GKD / 2));
      const int rem = t - op * (G48 * (GKD / 2));
      const int c = rem / (GKD / 2), q = rem - c * (GKD / 2);
      const double* src = op ? B : A;
      const int ld = op ? ldb : lda;
      const int cc = op ? cb : ca;
      double* dst = (op ? Bs[buf] : As[buf]) + g48d_off(c, 2 * q);
      const int k = k0 + 2 * q;
      const int nv = (c < cc) ? max(0, min(2, k_end - k)) : 0;
      const double* g = nv ? src + (size_t)c * ld + k : src;
      if (vec) {
        cp_async16(dst, g, 8 * nv);
      } else {
        const float* gf = reinterpret_cast<const float*>(g);
        const float* sf = reinterpret_cast<const float*>(src);
        float* df = reinterpret_cast<float*>(dst);
#pragma unroll
        for (int u = 0; u < 4; ++u) cp_async4(df + u, u < 2 * nv ? gf + u : sf, u < 2 * nv ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
  const int nst = (k_end > k_beg) ? (k_end - k_beg + GKD - 1) / GKD : 0;
  if (nst > 0) load_stage(0, k_beg);
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) {
      load_stage((st + 1) & 1, k_beg + (st + 1) * GKD);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // split the stage into FP32 parts, transposed to [row][column]
    for (int t = threadIdx.x; t < 2 * G48 * GKD; t += blockDim.x) {
      const int op = t / (G48 * GKD);
      const int rem = t - op * (G48 * GKD);
      const int c = rem / GKD, r = rem - c * GKD;
      const double x = (op ? Bs[st & 1] : As[st & 1])[g48d_off(c, r)];
      const float h = __double2float_rn(x);
      const float l = __double2float_rn(x - (double)h);
      (op ? Bh : Ah)[r][c] = h;
      (op ? Bl : Al)[r][c] = l;
    }
    __syncthreads();
#pragma unroll 2
    for (int r = 0; r < GKD; ++r) {
      const float4 ah = *reinterpret_cast<const float4*>(&Ah[r][ty * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&Al[r][ty * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[r][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[r][tx * 4]);
      const float a_h[4] = {ah.x, ah.y, ah.z, ah.w}, a_l[4] = {al.x, al.y, al.z, al.w};
      const float b_h[4] = {bh.x, bh.y, bh.z, bh.w}, b_l[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = __fmul_rn(a_h[i], b_h[j]);              // never contracted into the sum
          const float pe = fmaf(a_h[i], b_h[j], -p);           // exact: p + pe = a_h b_h
          const float cr = fmaf(a_h[i], b_l[j], a_l[i] * b_h[j]);
          const float s = sh[i][j] + p;                          // two-sum of sh and p
          const float bp = s - sh[i][j];
          const float err = (sh[i][j] - (s - bp)) + (p - bp);
          sh[i][j] = s;
          sl[i][j] += err + (pe + cr);
        }
    }
    // renormalise the pairs: the low part stays within a few units of the
    // high part's last place, so its own rounding stays at ~2^-48 of it
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float t = sh[i][j] + sl[i][j];
        sl[i][j] -= t - sh[i][j];
        sh[i][j] = t;
      }
    __syncthreads();
  }
  double* out = partial + blockIdx.z * pstride + ((size_t)blockIdx.y * gridDim.x + pair) * (TILE * TILE);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * TILE + tx * 4 + j] = (double)sh[i][j] + (double)sl[i][j];
}

template <class real>
__global__ void gram_reduce_kernel(const ElemDev<real>* __restrict__ elems, GramJob<real> job,
                                   const double* __restrict__ partial, size_t pstride, int nchunk,
                                   int tiles_a, int tiles_b) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int ntile = tiles_a * tiles_b;
  const int pair = blockIdx.x / ntile;
  const int t = blockIdx.x - pair * ntile;
  const int ta = t / tiles_b, tb = t - ta * tiles_b;
  if (job.needs_p[pair] && !e.state[ST_HAS_P]) return;
  const int ca = job.ncols_a > 0 ? job.ncols_a : e.m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : e.m;
  const int a0 = ta * TILE, b0 = tb * TILE;
  if (a0 >= ca || b0 >= cb) return;
  double* out;
  int ld;
  switch (job.out_id[pair]) {
    case OUT_GRAM_A: out = e.gram; ld = job.ld_out > 0 ? job.ld_out : 3 * e.m; break;
    case OUT_GRAM_B: out = e.gram + (size_t)9 * e.m * e.m; ld = job.ld_out > 0 ? job.ld_out : 3 * e.m; break;
    case OUT_GXW: out = e.gxw; ld = job.ld_out > 0 ? job.ld_out : e.m; break;
    default: out = job.out_ptr; ld = job.ld_out; break;
  }
  const double* base = partial + blockIdx.z * pstride + (size_t)blockIdx.x * (TILE * TILE);
  const size_t cstride = (size_t)gridDim.x * (TILE * TILE);
  for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
    const int r = i / TILE, c = i - r * TILE;
    if (a0 + r >= ca || b0 + c >= cb) continue;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += base[ch * cstride + i];
    const int orow = job.brow[pair] * ca + a0 + r;
    const int ocol = job.bcol[pair] * cb + b0 + c;
    out[orow + (size_t)ocol * ld] = s;
  }
}

// grid: (ceil(rows/64), ceil(ncols/64), nel); block 256.  Thread (tx, ty)
// owns rows tx + 16 i and columns ty * 4 + j of the 64 x 64 output tile.
template <class real>
__global__ void __launch_bounds__(256) tsmm_kernel(const ElemDev<real>* __restrict__ elems,
                                                   TsmmJob<real> job) {
  __shared__ real Ss[KU][TILE + 4];
  __shared__ real Ys[KU][TILE + 4];
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int nc = job.ncols > 0 ? job.ncols : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const int r0 = blockIdx.x * TILE, c0 = blockIdx.y * TILE;
  if (r0 >= rows || c0 >= nc) return;
  const double* Y;
  int ldy;
  switch (job.y_id) {
    case Y_RR: Y = e.Y; ldy = job.ldy > 0 ? job.ldy : 3 * e.m; break;
    case Y_GXW: Y = e.gxw; ldy = job.ldy > 0 ? job.ldy : e.m; break;
    default: Y = job.y_ptr; ldy = job.ldy; break;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  real acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  const int ycol0 = job.ycol * nc + c0;
  for (int in = 0; in < job.nin; ++in) {
    if (job.needs_p[in] && !e.state[ST_HAS_P]) continue;
    const real* S = resolve(e, job.in[in]);
    const int lds = ld_of(e, job.in[in], job.ld_in, rows);
    const int yrow0 = job.yrow[in] * nc;
    for (int k0 = 0; k0 < nc; k0 += KU) {
      for (int i = threadIdx.x; i < KU * TILE; i += blockDim.x) {
        const int kk = i / TILE, r = i - kk * TILE;
        const bool kin = k0 + kk < nc;
        Ss[kk][r] = (kin && r0 + r < rows) ? S[(size_t)(k0 + kk) * lds + r0 + r] : (real)0;
        Ys[kk][r] = (kin && c0 + r < nc) ? (real)Y[(yrow0 + k0 + kk) + (size_t)(ycol0 + r) * ldy] : (real)0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KU; ++kk) {
        real sv[4], yv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) sv[i] = Ss[kk][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) yv[j] = Ys[kk][ty * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += sv[i] * yv[j];
      }
      __syncthreads();
    }
  }
  real* O = resolve(e, job.out);
  const int ldo = ld_of(e, job.out, job.ld_in, rows);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int col = c0 + ty * 4 + j;
    if (col >= nc) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + tx + 16 * i;
      if (row >= rows) continue;
      real* o = O + (size_t)col * ldo + row;
      real v = (real)job.alpha * acc[i][j];
      if (job.beta != 0.0) v += (real)job.beta * *o;
      *o = v;
    }
  }
}

// FP64 block update in double-float arithmetic (the mixed form's FP64 stage):
// the tiling of tsmm_kernel, with every staged block and coefficient value
// split into FP32 parts (x = xh + xl) and each output accumulated as a
// (hi, lo) FP32 pair: exact leading products by FMA, cross terms, a two-sum
// per product (~2^-44 relative, at FP32-pipe rates).  alpha and beta are
// applied in FP64 to the pair's sum.
__global__ void __launch_bounds__(256) tsmm_df_kernel(const ElemDev<double>* __restrict__ elems,
                                                       TsmmJob<double> job) {
  __shared__ float Sh[KU][TILE + 4], Sl[KU][TILE + 4];
  __shared__ float Yh[KU][TILE + 4], Yl[KU][TILE + 4];
  const ElemDev<double>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int nc = job.ncols > 0 ? job.ncols : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const int r0 = blockIdx.x * TILE, c0 = blockIdx.y * TILE;
  if (r0 >= rows || c0 >= nc) return;
  const double* Y;
  int ldy;
  switch (job.y_id) {
    case Y_RR: Y = e.Y; ldy = job.ldy > 0 ? job.ldy : 3 * e.m; break;
    case Y_GXW: Y = e.gxw; ldy = job.ldy > 0 ? job.ldy : e.m; break;
    default: Y = job.y_ptr; ldy = job.ldy; break;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float ah[4][4], al[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ah[i][j] = al[i][j] = 0.f;
  const int ycol0 = job.ycol * nc + c0;
  for (int in = 0; in < job.nin; ++in) {
    if (job.needs_p[in] && !e.state[ST_HAS_P]) continue;
    const double* S = resolve(e, job.in[in]);
    const int lds = ld_of(e, job.in[in], job.ld_in, rows);
    const int yrow0 = job.yrow[in] * nc;
    for (int k0 = 0; k0 < nc; k0 += KU) {
      for (int i = threadIdx.x; i < KU * TILE; i += blockDim.x) {
        const int kk = i / TILE, r = i - kk * TILE;
        const bool kin = k0 + kk < nc;
        const double sv = (kin && r0 + r < rows) ? S[(size_t)(k0 + kk) * lds + r0 + r] : 0.0;
        const double yv = (kin && c0 + r < nc) ? Y[(yrow0 + k0 + kk) + (size_t)(ycol0 + r) * ldy] : 0.0;
        const float svh = __double2float_rn(sv), yvh = __double2float_rn(yv);
        Sh[kk][r] = svh;
        Sl[kk][r] = __double2float_rn(sv - (double)svh);
        Yh[kk][r] = yvh;
        Yl[kk][r] = __double2float_rn(yv - (double)yvh);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KU; ++kk) {
        float sh[4], sl[4], yh[4], yl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          sh[i] = Sh[kk][tx + 16 * i];
          sl[i] = Sl[kk][tx + 16 * i];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          yh[j] = Yh[kk][ty * 4 + j];
          yl[j] = Yl[kk][ty * 4 + j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float p = __fmul_rn(sh[i], yh[j]);  // never contracted into the sum
            const float pe = fmaf(sh[i], yh[j], -p);
            const float cr = fmaf(sh[i], yl[j], sl[i] * yh[j]);
            const float t = ah[i][j] + p;
            const float bp = t - ah[i][j];
            const float err = (ah[i][j] - (t - bp)) + (p - bp);
            ah[i][j] = t;
            al[i][j] += err + (pe + cr);
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float t = ah[i][j] + al[i][j];
          al[i][j] -= t - ah[i][j];
          ah[i][j] = t;
        }
      __syncthreads();
    }
  }
  double* O = resolve(e, job.out);
  const int ldo = ld_of(e, job.out, job.ld_in, rows);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int col = c0 + ty * 4 + j;
    if (col >= nc) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + tx + 16 * i;
      if (row >= rows) continue;
      double* o = O + (size_t)col * ldo + row;
      double v = job.alpha * ((double)ah[i][j] + (double)al[i][j]);
      if (job.beta != 0.0) v += job.beta * *o;
      *o = v;
    }
  }
}

// FP32 block update out = alpha sum_i in_i Y_i + beta out (and optionally
// out2 = the partial sum over inputs i >= from2) for up to 48 output
// columns per CTA tile: 128 rows x 48 columns per CTA of 128 threads, each
// thread 4 rows x 12 columns.  Y (all inputs' rows x 48 columns) is
// converted to FP32 into shared memory once per CTA; the input rows stream
// through a double-buffered cp.async stage of TK k-values x 128 rows.
// grid: (row-tile groups, column tiles, nel); block 128.
constexpr int TS_THREADS = 128;
constexpr int TS_CT = 48;
constexpr int TS_TR = 128;
constexpr int TS_TK = 16;

__global__ void __launch_bounds__(TS_THREADS, 4) tsmm_rows_kernel(const ElemDev<float>* __restrict__ elems,
                                                               TsmmJob<float> job) {
  extern __shared__ __align__(16) float tsm[];
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int nc = job.ncols > 0 ? job.ncols : e.m;
  const int rows = job.rows > 0 ? job.rows : e.ng;
  const int c0 = blockIdx.y * TS_CT;
  if (c0 >= nc) return;
  const double* Y;
  int ldy;
  switch (job.y_id) {
    case Y_RR: Y = e.Y; ldy = job.ldy > 0 ? job.ldy : 3 * e.m; break;
    case Y_GXW: Y = e.gxw; ldy = job.ldy > 0 ? job.ldy : e.m; break;
    default: Y = job.y_ptr; ldy = job.ldy; break;
  }
  const float* Yf = (job.y_id == Y_RR) ? e.Yf : nullptr;  // FP32 copy written by Rayleigh-Ritz
  const bool has_p = e.state[ST_HAS_P] != 0;
  const int ycol0 = job.ycol * nc + c0;
  const int ktot = job.nin * nc;
  float* ys = tsm;                                   // ktot x TS_CT
  float* ss = tsm + (size_t)ktot * TS_CT;            // 2 x TS_TK x TS_TR
  for (int t = threadIdx.x; t < ktot * TS_CT; t += blockDim.x) {
    const int c = t / ktot, kk = t - c * ktot;
    const int in = kk / nc, k = kk - in * nc;
    float v = 0.f;
    if (c0 + c < nc) {
      const size_t yi = (job.yrow[in] * nc + k) + (size_t)(ycol0 + c) * ldy;
      v = Yf ? Yf[yi] : (float)Y[yi];
    }
    ys[kk * TS_CT + c] = v;
  }
  // inputs in the order they are summed (last first), P skipped without P
  int act[3], nact = 0;
  for (int in = job.nin - 1; in >= 0; --in)
    if (!(job.needs_p[in] && !has_p)) act[nact++] = in;
  // out2 is complete after the last active input with index >= from2
  int q2 = -1;
  for (int q = 0; q < nact; ++q)
    if (job.from2 >= 0 && act[q] >= job.from2) q2 = q;
  const int cpi = (nc + TS_TK - 1) / TS_TK;  // stages per input
  const int nstage = nact * cpi;
  const int tr = threadIdx.x >> 2, tc = threadIdx.x & 3;
  const int ncol = min(TS_CT, nc - c0);
  const float alpha = (float)job.alpha, beta = (float)job.beta;
  float* O = resolve(e, job.out);
  const int ldo = ld_of(e, job.out, job.ld_in, rows);
  float* O2 = job.from2 >= 0 ? resolve(e, job.out2) : nullptr;
  const int ld2 = job.from2 >= 0 ? ld_of(e, job.out2, job.ld_in, rows) : 0;
  bool vec = true;
  for (int q = 0; q < nact; ++q) {
    const float* S = resolve(e, job.in[act[q]]);
    vec = vec && (ld_of(e, job.in[act[q]], job.ld_in, rows) & 3) == 0 && (((uintptr_t)S) & 15) == 0;
  }
  __syncthreads();
  for (int rt = blockIdx.x; rt * TS_TR < rows; rt += gridDim.x) {
    const int row0 = rt * TS_TR;
    auto load_stage = [&](int buf, int stg) {
      const int in = act[stg / cpi], k0 = (stg % cpi) * TS_TK;
      const float* S = resolve(e, job.in[in]);
      const int lds = ld_of(e, job.in[in], job.ld_in, rows);
      float* dst0 = ss + (size_t)buf * TS_TK * TS_TR;
      for (int t = threadIdx.x; t < TS_TK * (TS_TR / 4); t += blockDim.x) {
        const int kk = t / (TS_TR / 4), q = t - kk * (TS_TR / 4);
        const int k = k0 + kk, r = row0 + 4 * q;
        const int nv = (k < nc) ? max(0, min(4, rows - r)) : 0;
        const float* g = nv ? S + (size_t)k * lds + r : S;
        float* dst = dst0 + kk * TS_TR + 4 * q;
        if (vec) {
          cp_async16(dst, g, 4 * nv);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) cp_async4(dst + u, u < nv ? g + u : S, u < nv ? 4 : 0);
        }
      }
      cp_async_commit();
    };
    float acc[4][12];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[i][j] = 0.f;
    if (nstage > 0) load_stage(0, 0);
    for (int stg = 0; stg < nstage; ++stg) {
      if (stg + 1 < nstage) {
        load_stage((stg + 1) & 1, stg + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int in = act[stg / cpi], k0 = (stg % cpi) * TS_TK;
      const float* sb = ss + (size_t)(stg & 1) * TS_TK * TS_TR + 4 * tr;
      const float* yb = ys + ((size_t)in * nc + k0) * TS_CT + 12 * tc;
      const int kn = min(TS_TK, nc - k0);
#pragma unroll 4
      for (int kk = 0; kk < kn; ++kk) {
        const float4 s4 = *reinterpret_cast<const float4*>(sb + kk * TS_TR);
        const float4* y4 = reinterpret_cast<const float4*>(yb + (size_t)kk * TS_CT);
        const float4 ya = y4[0], yb4 = y4[1], yc = y4[2];
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
        const float yv[12] = {ya.x, ya.y, ya.z, ya.w, yb4.x, yb4.y, yb4.z, yb4.w, yc.x, yc.y, yc.z, yc.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 12; ++j) acc[i][j] = fmaf(sv[i], yv[j], acc[i][j]);
      }
      __syncthreads();
      if (O2 && (stg % cpi) == cpi - 1 && stg / cpi == q2) {
#pragma unroll
        for (int j = 0; j < 12; ++j) {
          const int c = 12 * tc + j;
          if (c >= ncol) continue;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = row0 + 4 * tr + i;
            if (r < rows) O2[(size_t)(c0 + c) * ld2 + r] = acc[i][j];
          }
        }
      }
    }
    if (O2 && q2 < 0) {
      // every input at or after from2 was skipped: out2 = 0
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        const int c = 12 * tc + j;
        if (c >= ncol) continue;
        for (int i = 0; i < 4; ++i) {
          const int r = row0 + 4 * tr + i;
          if (r < rows) O2[(size_t)(c0 + c) * ld2 + r] = 0.f;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const int c = 12 * tc + j;
      if (c >= ncol) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = row0 + 4 * tr + i;
        if (r < rows) {
          float* o = O + (size_t)(c0 + c) * ldo + r;
          *o = (beta == 0.f) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *o;
        }
      }
    }
  }
}

size_t tsmm_rows_smem(int nin, int nc) {
  return sizeof(float) * ((size_t)nin * nc * TS_CT + 2 * (size_t)TS_TK * TS_TR);
}

// R = HX - X diag(theta) into W; partial sums (r.r, x.x, x.Hx, x.V x).
template <class real>
__global__ void __launch_bounds__(256) residual_kernel(const ElemDev<real>* __restrict__ elems,
                                                       int nchunk) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int j = blockIdx.y;
  if (j >= e.m) return;
  const int kc = (((e.ng + nchunk - 1) / nchunk) + 3) & ~3;  // chunks of whole 16-byte groups
  const int beg = blockIdx.x * kc, end = min(e.ng, beg + kc);
  const real* X = cur_blk(e, BX) + (size_t)j * e.ng;
  const real* HX = cur_blk(e, BHX) + (size_t)j * e.ng;
  real* R = e.blk[BW][0] + (size_t)j * e.ng;
  const real th = (real)e.theta[j];
  real s[4] = {0, 0, 0, 0};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (sizeof(real) == sizeof(float)) {
    // FP32: 16-byte accesses where the columns allow, and a block reduction
    // in FP32 (the FP64 pipe of this part is ~55x slower; these are partial
    // sums of at most a few thousand terms, converted to FP64 per chunk)
    const bool vec = ((beg | end) & 3) == 0 && ((e.ng & 3) == 0) &&
                     ((((uintptr_t)X) | ((uintptr_t)HX) | ((uintptr_t)R) | ((uintptr_t)e.V)) & 15) == 0;
    if (vec) {
      const float4* X4 = reinterpret_cast<const float4*>(X);
      const float4* H4 = reinterpret_cast<const float4*>(HX);
      const float4* V4 = reinterpret_cast<const float4*>(e.V);
      float4* R4 = reinterpret_cast<float4*>(R);
#pragma unroll 2
      for (int i = (beg >> 2) + threadIdx.x; i < (end >> 2); i += blockDim.x) {
        const float4 x = X4[i], hx = H4[i], v = V4[i];
        const float4 r = make_float4(hx.x - th * x.x, hx.y - th * x.y, hx.z - th * x.z, hx.w - th * x.w);
        R4[i] = r;
        s[0] += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
        s[1] += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        s[2] += x.x * hx.x + x.y * hx.y + x.z * hx.z + x.w * hx.w;
        s[3] += v.x * x.x * x.x + v.y * x.y * x.y + v.z * x.z * x.z + v.w * x.w * x.w;
      }
    } else {
      for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const real x = X[i], hx = HX[i];
        const real r = hx - th * x;
        R[i] = r;
        s[0] += r * r;
        s[1] += x * x;
        s[2] += x * hx;
        s[3] += e.V[i] * x * x;
      }
    }
    __shared__ float redf[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float v = s[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) redf[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      float v = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += redf[threadIdx.x][w];
      e.rpart[((size_t)j * nchunk + blockIdx.x) * 4 + threadIdx.x] = (double)v;
    }
  } else {
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
      const real x = X[i], hx = HX[i];
      const real r = hx - th * x;
      R[i] = r;
      s[0] += r * r;
      s[1] += x * x;
      s[2] += x * hx;
      s[3] += e.V[i] * x * x;
    }
    __shared__ double red[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = warp_sum((double)s[q]);
      if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
      e.rpart[((size_t)j * nchunk + blockIdx.x) * 4 + threadIdx.x] = v;
    }
  }
}

// r.r of the W block per chunk of the residual kernel (same chunks, same
// grid), overwriting that kernel's first partial sum: the residual norm of
// the sphere-cutoff set is |P R|, taken after W = R was projected.  Sums in
// the working precision within a CTA (as the residual kernel), FP64 across.
template <class real>
__global__ void __launch_bounds__(256) rnorm_kernel(const ElemDev<real>* __restrict__ elems, int nchunk) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int j = blockIdx.y;
  if (j >= e.m) return;
  const int kc = (((e.ng + nchunk - 1) / nchunk) + 3) & ~3;
  const int beg = blockIdx.x * kc, end = min(e.ng, beg + kc);
  const real* R = e.blk[BW][0] + (size_t)j * e.ng;
  real s = 0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) s += R[i] * R[i];
  __shared__ real red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s = warp_sum(s);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    real v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    e.rpart[((size_t)j * nchunk + blockIdx.x) * 4] = (double)v;
  }
}

template <class real>
__global__ void post_residual_kernel(const ElemDev<real>* __restrict__ elems, int nchunk, int maxit) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  __shared__ double smax[256];
  __shared__ int sbad[256];
  double mx = 0.0;
  int bad = 0;
  for (int j = threadIdx.x; j < e.m; j += blockDim.x) {
    double s[4] = {0, 0, 0, 0};
    for (int c = 0; c < nchunk; ++c)
      for (int q = 0; q < 4; ++q) s[q] += e.rpart[((size_t)j * nchunk + c) * 4 + q];
    double nl = 0.0;
    for (int p = 0; p < e.n_proj; ++p) {
      const double c = (double)e.Ccoef[p + (size_t)j * e.n_proj];
      nl += e.p_gamma[p] * c * c;
    }
    const double res = sqrt(s[0] / s[1]);
    e.res[j] = res;
    // x.Hx was taken with H - sigma I
    e.tkin[j] = (s[2] + e.sigma[0] * s[1] - s[3] - nl) / s[1];
    if (!isfinite(res)) bad = 1;
    if (j < e.J) mx = fmax(mx, res);
  }
  smax[threadIdx.x] = mx;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < blockDim.x; ++t) {
      mx = fmax(mx, smax[t]);
      bad |= sbad[t];
    }
    int* st = e.state;
    if (bad) {
      st[ST_ERROR] |= ERR_NONFINITE;
      st[ST_ACTIVE] = 0;
    } else if (mx <= e.tol) {
      st[ST_CONVERGED] = 1;
      st[ST_ACTIVE] = 0;
    } else if (st[ST_ITER] >= maxit) {
      st[ST_ACTIVE] = 0;
    } else {
      st[ST_ITER] += 1;
    }
    if constexpr (sizeof(real) == sizeof(float)) {
      // Re-centre the spectral shift on the Ritz values once they have
      // settled: the Gram entries that carry the residual information
      // ((H - sigma) x_i against the basis) then shrink from |theta| to
      // |theta - sigma|, and with them the FP32 rounding of those sums.
      double d = 0.0;
      if (st[ST_ACTIVE] && mx < SHIFT_RES) {
        const double lo = e.theta[0], hi = e.theta[e.m - 1];
        const double mid = 0.5 * (lo + hi);
        if (fabs(mid) > 0.25 * (hi - lo) + 1e-3) d = mid;
      }
      e.sigma[1] = d;
      if (d != 0.0) {
        e.sigma[0] += d;
        for (int j = 0; j < e.m; ++j) e.theta[j] -= d;
      }
    }
  }
}

// After a change d of the shift: HX -= d X and HP -= d P, keeping the stored
// H-images equal to (H - sigma I) applied to their blocks.
template <class real>
__global__ void __launch_bounds__(256) shift_kernel(const ElemDev<real>* __restrict__ elems) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const double d = e.sigma[1];
  if (d == 0.0) return;
  const real dr = (real)d;
  const size_t n = (size_t)e.ng * e.m;
  const bool has_p = e.state[ST_HAS_P] != 0;
  real* hx = cur_blk(e, BHX);
  const real* x = cur_blk(e, BX);
  real* hp = cur_blk(e, BHP);
  const real* p = cur_blk(e, BP);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    hx[i] -= dr * x[i];
    if (has_p) hp[i] -= dr * p[i];
  }
}

// theta_j = 0 (mode 0) or the Rayleigh quotient x.Hx / x.x from the residual
// partial sums (mode 1), for every column of every active element.
template <class real>
__global__ void theta_kernel(const ElemDev<real>* __restrict__ elems, int nchunk, int mode) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  for (int j = threadIdx.x; j < e.m; j += blockDim.x) {
    if (mode == 0) {
      e.theta[j] = 0.0;
      continue;
    }
    double xx = 0.0, xhx = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      xx += e.rpart[((size_t)j * nchunk + c) * 4 + 1];
      xhx += e.rpart[((size_t)j * nchunk + c) * 4 + 2];
    }
    e.theta[j] = xhx / xx;
  }
}

template <class real>
__global__ void iter_finish_kernel(const ElemDev<real>* __restrict__ elems, int nel, int set_p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nel) return;
  int* st = elems[i].state;
  if (!st[ST_ACTIVE]) return;
  st[ST_PARITY] ^= 1;
  if (st[ST_RESTART]) {
    // restarted this iteration: P' = 0, the next pencil is [X W]
    st[ST_HAS_P] = 0;
    st[ST_RESTART] = 0;
  } else if (set_p) {
    st[ST_HAS_P] = 1;
  }
}

// Uniform in [-1, 1) from a 32-bit integer mix of (a, b).
__device__ __forceinline__ float mix_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u + b * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

// Restart of an element whose Rayleigh-Ritz found no usable pencil (X' = X
// was written): add a seeded perturbation of relative size RESTART_AMP to
// every column of X' (entries of a unit column are ~1/sqrt(N_g)), which
// makes nearly dependent columns independent again; H X' is computed from
// the perturbed block, and P is dropped for the next iteration.
constexpr float RESTART_AMP = 0.03f;

template <class real>
__global__ void restart_kernel(const ElemDev<real>* __restrict__ elems) {
  const ElemDev<real>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE] || !e.state[ST_RESTART]) return;
  real* x = next_blk(e, BX);
  const size_t n = (size_t)e.ng * e.m;
  const float amp = RESTART_AMP * rsqrtf((float)e.ng);
  const unsigned seed = 0x51EDu * (unsigned)(blockIdx.z + 1) + 0x2545F491u * (unsigned)e.state[ST_NRESTART];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += (real)(amp * mix_unit((unsigned)i, seed));
}

}  // namespace

template <class real>
void launch_gram(const Batch<real>& b, const GramJob<real>& job, double* partial, size_t partial_cap,
                 cudaStream_t st) {
  const BatchShape& s = b.s;
  const int ca = job.ncols_a > 0 ? job.ncols_a : s.max_m;
  const int cb = job.ncols_b > 0 ? job.ncols_b : s.max_m;
  const int rows = job.rows > 0 ? job.rows : s.max_ng;
  const int tiles_a = (ca + TILE - 1) / TILE, tiles_b = (cb + TILE - 1) / TILE;
  const int ny = job.npairs * tiles_a * tiles_b;
  // per-element partial storage: nchunk * ny tiles
  int kchunk = 2048;
  int nchunk = (rows + kchunk - 1) / kchunk;
  while ((size_t)nchunk * ny * TILE * TILE * s.nel > partial_cap && kchunk < (1 << 30)) {
    kchunk *= 2;
    nchunk = (rows + kchunk - 1) / kchunk;
  }
  const size_t pstride = (size_t)nchunk * ny * TILE * TILE;
  if (std::is_same<real, float>::value && ca <= G48 && cb <= G48) {
    gram48_kernel<<<dim3(ny, nchunk, s.nel), 144, 0, st>>>(
        reinterpret_cast<const ElemDev<float>*>(b.d_elems), *reinterpret_cast<const GramJob<float>*>(&job), partial,
        pstride, kchunk);
  } else if (std::is_same<real, double>::value && ca <= G48 && cb <= G48 && s.dfloat) {
    gram48df_kernel<<<dim3(ny, nchunk, s.nel), 144, 0, st>>>(
        reinterpret_cast<const ElemDev<double>*>(b.d_elems), *reinterpret_cast<const GramJob<double>*>(&job),
        partial, pstride, kchunk);
  } else if (std::is_same<real, double>::value && ca <= G48 && cb <= G48) {
    gram48d_kernel<<<dim3(ny, nchunk, s.nel), 144, 0, st>>>(
        reinterpret_cast<const ElemDev<double>*>(b.d_elems), *reinterpret_cast<const GramJob<double>*>(&job),
        partial, pstride, kchunk);
  } else {
    gram_kernel<real><<<dim3(nchunk, ny, s.nel), 256, 0, st>>>(b.d_elems, job, partial, pstride, kchunk,
                                                               tiles_a, tiles_b);
  }
  gram_reduce_kernel<real><<<dim3(ny, 1, s.nel), 256, 0, st>>>(b.d_elems, job, partial, pstride, nchunk,
                                                               tiles_a, tiles_b);
}

template <class real>
void launch_tsmm(const Batch<real>& b, const TsmmJob<real>& job, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = job.ncols > 0 ? job.ncols : s.max_m;
  if constexpr (std::is_same<real, float>::value) {
    const size_t smem = tsmm_rows_smem(job.nin, nc);
    if (smem <= 160 * 1024) {
      const int rows = job.rows > 0 ? job.rows : s.max_ng;
      // s.tsmm_tiles 128-row tiles per CTA (default 8, or the autotuner's
      // choice): the Y staging (ktot x 48 coefficients per CTA) is amortised;
      // 1.87 ms against 2.24 ms with two tiles on the 36-element monolayer
      const int tpc = s.tsmm_tiles > 0 ? s.tsmm_tiles : 8;
      const int gx = std::max(1, (rows + tpc * TS_TR - 1) / (tpc * TS_TR));
      tsmm_rows_kernel<<<dim3(gx, (nc + TS_CT - 1) / TS_CT, s.nel), TS_THREADS, smem, st>>>(b.d_elems, job);
      return;
    }
  }
  const int rows = job.rows > 0 ? job.rows : s.max_ng;
  if constexpr (std::is_same<real, double>::value) {
    if (s.dfloat) {
      tsmm_df_kernel<<<dim3((rows + TILE - 1) / TILE, (nc + TILE - 1) / TILE, s.nel), 256, 0, st>>>(b.d_elems,
                                                                                                  job);
      return;
    }
  }
  tsmm_kernel<real><<<dim3((rows + TILE - 1) / TILE, (nc + TILE - 1) / TILE, s.nel), 256, 0, st>>>(
      b.d_elems, job);
}

template <class real>
void launch_residual(const Batch<real>& b, int nchunk, cudaStream_t st) {
  residual_kernel<real><<<dim3(nchunk, b.s.max_m, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk);
}

template <class real>
void launch_post_residual(const Batch<real>& b, int nchunk, int maxit, cudaStream_t st) {
  post_residual_kernel<real><<<dim3(1, 1, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk, maxit);
}

void launch_rnorm(const Batch<double>& b, int nchunk, cudaStream_t st) {
  rnorm_kernel<double><<<dim3(nchunk, b.s.max_m, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk);
}
void launch_rnorm(const Batch<float>& b, int nchunk, cudaStream_t st) {
  rnorm_kernel<float><<<dim3(nchunk, b.s.max_m, b.s.nel), 256, 0, st>>>(b.d_elems, nchunk);
}

template <class real>
void launch_shift(const Batch<real>& b, cudaStream_t st) {
  const int per_elem = std::max(8, 1216 / std::max(1, b.s.nel));
  shift_kernel<real><<<dim3(per_elem, 1, b.s.nel), 256, 0, st>>>(b.d_elems);
}

template <class real>
void launch_theta(const Batch<real>& b, int nchunk, int mode, cudaStream_t st) {
  theta_kernel<real><<<dim3(1, 1, b.s.nel), 128, 0, st>>>(b.d_elems, nchunk, mode);
}

template <class real>
void launch_restart(const Batch<real>& b, cudaStream_t st) {
  restart_kernel<real><<<dim3(64, 1, b.s.nel), 256, 0, st>>>(b.d_elems);
}

template <class real>
void launch_iter_finish(const Batch<real>& b, int set_p, cudaStream_t st) {
  iter_finish_kernel<real><<<(b.s.nel + 127) / 128, 128, 0, st>>>(b.d_elems, b.s.nel, set_p);
}

void init_blas_kernels() { opt_in_dynamic_smem((const void*)tsmm_rows_kernel); }

#define DGDFT_INST(real)                                                                             \
  template void launch_gram<real>(const Batch<real>&, const GramJob<real>&, double*, size_t,         \
                                  cudaStream_t);                                                     \
  template void launch_tsmm<real>(const Batch<real>&, const TsmmJob<real>&, cudaStream_t);           \
  template void launch_residual<real>(const Batch<real>&, int, cudaStream_t);                        \
  template void launch_post_residual<real>(const Batch<real>&, int, int, cudaStream_t);              \
  template void launch_iter_finish<real>(const Batch<real>&, int, cudaStream_t);                    \
  template void launch_restart<real>(const Batch<real>&, cudaStream_t);                              \
  template void launch_theta<real>(const Batch<real>&, int, int, cudaStream_t);                     \
  template void launch_shift<real>(const Batch<real>&, cudaStream_t);
DGDFT_INST(double)
DGDFT_INST(float)
#undef DGDFT_INST

}  // namespace dgdft
