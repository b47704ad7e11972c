// Tensor-core Gram products for the FP32 stage (Sec. II.B, operation 2).
//
// C = U^T V over the N_g rows of each element, where U is a concatenation of
// up to 6 column blocks (the MMA M side, padded to 128) and V of up to 3
// blocks (the N side).  Every FP32 value x is split into bf16 parts
// hi = bf16(x), lo = bf16(x - hi) and the product (hi + lo)(hi + lo) is
// accumulated in FP32 in tensor memory as four bf16 products.  The lo*lo
// term is kept: it is always positive on the diagonal of S^T S, so dropping
// it would bias the overlap matrix by ~2^-18 relative; what remains is the
// random rounding of lo (~2^-17 relative per value).
//
// Each CTA (128 threads) owns one 128-row M tile and one chunk of rows:
//   * threads load FP32 from HBM (coalesced along rows), split, and store the
//     bf16 parts into shared memory in the 128-byte-swizzled K-major layout;
//   * one thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32, M = 128,
//     K = 16 per instruction) into a TMEM accumulator of N columns; a
//     tcgen05.commit per chunk arrives on an mbarrier, so the next chunk's
//     loads overlap the MMAs of the previous one (two smem stages);
//   * the epilogue reads TMEM with tcgen05.ld and writes FP64 partial sums,
//     reduced over chunks in a fixed order by a second kernel.
// Every mbarrier wait is bounded: on expiry the kernel records an error in
// the element's state word, drains, frees TMEM and returns.
#include <cuda_bf16.h>

#include "internal.h"

namespace dgdft {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KC = 64;                    // rows (K) per stage: one 128-byte bf16 row
constexpr int TC_THREADS = 256;
constexpr int TC_NMAX = 256;                 // accumulator columns (N <= 256)
constexpr int A_BYTES = TC_M * TC_KC * 2;    // one bf16 part of the A tile: 16 KB
constexpr uint32_t SPIN_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < SPIN_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  // tcgen05 shared-memory descriptor, K-major, 128-byte swizzle:
  // start >> 4 (bits 0-13), LBO = 1 (16-29, unused for swizzled K-major),
  // SBO = 1024 B between 8-row groups (32-45), fixed 0b001 (46-48),
  // swizzle mode 2 = 128B (61-63).
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ uint32_t idesc_bf16_f32(int M, int N) {
  // kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16
  // (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of bf16 element (row r, k) in a K-major 128B-swizzled tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

struct TcSide {
  int nblk;
  int cols;               // columns per block (<= 0: the element's m)
  int sel[6];
  int needs_p[6];
  const float* ptr[6];    // explicit block (ld = the element's N_g) or nullptr
};

struct TcGramArgs {
  TcSide a, b;   // U blocks (M side), V blocks (N side), each m columns
  int tiles_m;   // number of 128-row M tiles
  int kchunk;    // rows per CTA (multiple of TC_KC)
  size_t pstride;  // per-element partial stride (doubles)
  double* out;     // explicit output (out_mode 2), p x q column-major
};

__device__ __forceinline__ int side_cols(const ElemDev<float>& e, const TcSide& s) {
  return s.cols > 0 ? s.cols : e.m;
}

// Resolve the column `col` of a concatenated side to a pointer (nullptr for
// padding or an absent P block).
__device__ __forceinline__ const float* side_col(const ElemDev<float>& e, const TcSide& s, int col) {
  const int cols = side_cols(e, s);
  const int b = col / cols;
  if (b >= s.nblk) return nullptr;
  if (s.needs_p[b] && !e.state[ST_HAS_P]) return nullptr;
  const float* base = s.ptr[b] ? s.ptr[b] : cur_blk(e, s.sel[b]);
  return base + (size_t)(col - b * cols) * e.ng;
}

// Split two consecutive-k values (k even) and store both parts as packed pairs.
__device__ __forceinline__ void split_store2(unsigned char* hi, unsigned char* lo, int r, int k, float x0,
                                             float x1) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
  const uint32_t off = sw128_off(r, k);
  __nv_bfloat162 hp, lp;
  hp.x = h0;
  hp.y = h1;
  lp.x = l0;
  lp.y = l1;
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = hp;
  *reinterpret_cast<__nv_bfloat162*>(lo + off) = lp;
}

// grid: (nchunk, tiles_m, nel); dynamic smem: 2 stages x (A hi/lo + B hi/lo) + 1 KB.
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gram_kernel(const ElemDev<float>* __restrict__ elems, TcGramArgs args, double* __restrict__ partial) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int M_total = args.a.nblk * side_cols(e, args.a);
  const int N_real = args.b.nblk * side_cols(e, args.b);
  const int N = (N_real + 15) & ~15;        // MMA N: multiple of 16 for M = 128, <= 256
  const int mt = blockIdx.y;
  if (mt * TC_M >= M_total) return;
  const int rows = e.ng;
  // float2 loads need every column to start on an 8-byte boundary: even N_g
  // (always true for solver blocks, nx being even) and k0 even
  const bool vec2 = (rows & 1) == 0;
  const int k_beg = blockIdx.x * args.kchunk;
  const int k_end = min(rows, k_beg + args.kchunk);
  const int nsteps = (k_end > k_beg) ? (k_end - k_beg + TC_KC - 1) / TC_KC : 0;
  // shared layout (1024-aligned): per stage A_hi, A_lo (16 KB each), B_hi, B_lo (N*128 B each)
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int b_bytes = ((N + 7) / 8) * 1024;
  const int stage_bytes = 2 * A_BYTES + 2 * b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_NMAX)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16_f32(TC_M, N);

  for (int c = 0; c < nsteps; ++c) {
    const int s = c & 1;
    unsigned char* st = base + s * stage_bytes;
    unsigned char* a_hi = st;
    unsigned char* a_lo = st + A_BYTES;
    unsigned char* b_hi = st + 2 * A_BYTES;
    unsigned char* b_lo = b_hi + b_bytes;
    if (c >= 2) {
      // the MMAs that read this stage two chunks ago must be complete
      if (!mbar_wait(&bars[s], ((c >> 1) - 1) & 1)) atomicOr(&abort_flag, 1);
    }
    __syncthreads();
    if (abort_flag) break;
    const int k0 = k_beg + c * TC_KC;
    // A tile (128 columns) then B tile (N columns), 64 rows each: every warp
    // takes columns warp, warp + NW, ...; lanes read two consecutive rows of a
    // column.  Eight columns' loads are issued before any is converted so the
    // loads overlap instead of forming a dependent chain.
    constexpr int NW = TC_THREADS / 32;
    constexpr int BATCH = 8;
    const int k = 2 * lane;
    const int g = k0 + k;
    for (int side = 0; side < 2; ++side) {
      const int ncol = side ? N : TC_M;
      unsigned char* hi = side ? b_hi : a_hi;
      unsigned char* lo = side ? b_lo : a_lo;
      for (int q0 = warp; q0 < ncol; q0 += NW * BATCH) {
        float2 v[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
          const int q = q0 + u * NW;
          const float* src = nullptr;
          if (q < ncol) {
            if (side) {
              src = (q < N_real) ? side_col(e, args.b, q) : nullptr;
            } else {
              const int col = mt * TC_M + q;
              src = (col < M_total) ? side_col(e, args.a, col) : nullptr;
            }
          }
          v[u] = make_float2(0.f, 0.f);
          if (src) {
            if (vec2 && g + 1 < k_end) {
              v[u] = *reinterpret_cast<const float2*>(src + g);
            } else {
              if (g < k_end) v[u].x = src[g];
              if (g + 1 < k_end) v[u].y = src[g + 1];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
          const int q = q0 + u * NW;
          if (q < ncol) split_store2(hi, lo, q, k, v[u].x, v[u].y);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint32_t koff = kk * 32;  // 16 bf16 = 32 bytes along the swizzled row
        const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, sw128_desc(ah + koff), sw128_desc(bh + koff), idesc, acc0);
        mma_bf16(tmem, sw128_desc(ah + koff), sw128_desc(bl + koff), idesc, 1u);
        mma_bf16(tmem, sw128_desc(al + koff), sw128_desc(bh + koff), idesc, 1u);
        mma_bf16(tmem, sw128_desc(al + koff), sw128_desc(bl + koff), idesc, 1u);
      }
      mma_commit(&bars[s]);
    }
  }
  // drain: the last commit covers every MMA issued before it
  bool ok = !abort_flag;
  if (nsteps > 0) {
    const int last = nsteps - 1;
    if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  double* out = partial + blockIdx.z * args.pstride +
                ((size_t)blockIdx.x * args.tiles_m + mt) * ((size_t)TC_M * TC_NMAX);
  if (ok) {
    // a warp reads the TMEM lanes of its quarter (warp % 4); warps w and w + 4
    // take alternate 16-column groups
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;  // TMEM lane = M index within the tile
    for (int c0 = 16 * half; c0 < N; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) out[(size_t)row * TC_NMAX + c0 + j] = (nsteps > 0) ? (double)v[j] : 0.0;
    }
  } else if (tid == 0) {
    atomicOr(&e.state[ST_ERROR], ERR_EIG);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NMAX) : "memory");
}

// Sum the chunk partials and scatter C = [U blocks]^T [V blocks] into the
// element's Gram storage.  out_mode 0: LOBPCG (U = [S HS], V = S) -> A and B
// of the 3m pencil; out_mode 1: U = W, V = X -> gxw (X^T W).
__global__ void tc_gram_reduce_kernel(const ElemDev<float>* __restrict__ elems, TcGramArgs args,
                                      const double* __restrict__ partial, int nchunk, int out_mode) {
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int m = e.m;
  const int M_total = args.a.nblk * side_cols(e, args.a), N = args.b.nblk * side_cols(e, args.b);
  const double* base = partial + blockIdx.z * args.pstride;
  const size_t tile = (size_t)TC_M * TC_NMAX;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M_total * N; idx += gridDim.x * blockDim.x) {
    const int r = idx / N, c = idx - r * N;
    const int mt = r / TC_M, rr = r - mt * TC_M;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += base[((size_t)ch * args.tiles_m + mt) * tile + (size_t)rr * TC_NMAX + c];
    if (out_mode == 0) {
      const int ld = 3 * m;
      if (r < 3 * m) {
        e.gram[(size_t)9 * m * m + c + (size_t)r * ld] = s;  // B(c, r) = S_c . S_r
      } else {
        // A(j, c) = (HS)_j . S_c: in the upper block triangle H falls on the
        // earlier block, whose H-image after the shift is the small one
        e.gram[(r - 3 * m) + (size_t)c * ld] = s;
      }
    } else if (out_mode == 1) {
      e.gxw[c + (size_t)r * m] = s;  // (X^T W)(c, r) = X_c . W_r
    } else {
      args.out[r + (size_t)c * M_total] = s;  // C = U^T V, p x q
    }
  }
}

}  // namespace

size_t tc_gram_smem_bytes(int n_cols) {
  const int b_bytes = ((n_cols + 7) / 8) * 1024;
  return 2 * (2 * (size_t)A_BYTES + 2 * (size_t)b_bytes) + 1024;
}

void init_tc_gram_kernel() {
  opt_in_dynamic_smem((const void*)tc_gram_kernel);
}

// LOBPCG Gram blocks of the FP32 stage: mode 0 -> A, B from [S HS]^T S;
// mode 1 -> X^T W.  `partial` holds nel * nchunk * tiles_m * 128 * 256 doubles.
void launch_tc_gram(const Batch<float>& b, int mode, double* partial, size_t partial_cap, cudaStream_t st) {
  TcGramArgs a{};
  if (mode == 0) {
    const int sa[6] = {BX, BW, BP, BHX, BHW, BHP};
    a.a.nblk = 6;
    for (int i = 0; i < 6; ++i) {
      a.a.sel[i] = sa[i];
      a.a.needs_p[i] = (sa[i] == BP || sa[i] == BHP);
    }
    a.b.nblk = 3;
    const int sb[3] = {BX, BW, BP};
    for (int i = 0; i < 3; ++i) {
      a.b.sel[i] = sb[i];
      a.b.needs_p[i] = (sb[i] == BP);
    }
  } else {
    a.a.nblk = 1;
    a.a.sel[0] = BW;
    a.a.needs_p[0] = 0;
    a.b.nblk = 1;
    a.b.sel[0] = BX;
    a.b.needs_p[0] = 0;
  }
  a.a.cols = a.b.cols = 0;
  for (int i = 0; i < 6; ++i) a.a.ptr[i] = a.b.ptr[i] = nullptr;
  a.out = nullptr;
  const int m = b.s.max_m;
  a.tiles_m = (a.a.nblk * m + TC_M - 1) / TC_M;
  int kchunk = 2048;
  int nchunk = (b.s.max_ng + kchunk - 1) / kchunk;
  while ((size_t)nchunk * a.tiles_m * TC_M * TC_NMAX * b.s.nel > partial_cap) {
    kchunk *= 2;
    nchunk = (b.s.max_ng + kchunk - 1) / kchunk;
  }
  a.kchunk = kchunk;
  a.pstride = (size_t)nchunk * a.tiles_m * TC_M * TC_NMAX;
  const size_t smem = tc_gram_smem_bytes(((a.b.nblk * m) + 15) & ~15);
  tc_gram_kernel<<<dim3(nchunk, a.tiles_m, b.s.nel), TC_THREADS, smem, st>>>(b.d_elems, a, partial);
  const int total = a.a.nblk * m * a.b.nblk * m;
  tc_gram_reduce_kernel<<<dim3((total + 255) / 256, 1, b.s.nel), 256, 0, st>>>(b.d_elems, a, partial, nchunk,
                                                                                mode);
}

// C = U^T V for explicit FP32 blocks (single element view with ng rows):
// U is ng x p, V is ng x q, p, q <= 256 and q <= 256; C is p x q (FP64).
void launch_tc_gram_ptrs(const Batch<float>& b, const float* u, int p, const float* v, int q, int ng,
                         double* c, double* partial, size_t partial_cap, cudaStream_t st) {
  TcGramArgs a{};
  a.a.nblk = 1;
  a.a.cols = p;
  a.a.ptr[0] = u;
  a.a.needs_p[0] = 0;
  a.b.nblk = 1;
  a.b.cols = q;
  a.b.ptr[0] = v;
  a.b.needs_p[0] = 0;
  a.out = c;
  a.tiles_m = (p + TC_M - 1) / TC_M;
  int kchunk = 2048;
  int nchunk = (ng + kchunk - 1) / kchunk;
  while ((size_t)nchunk * a.tiles_m * TC_M * TC_NMAX > partial_cap) {
    kchunk *= 2;
    nchunk = (ng + kchunk - 1) / kchunk;
  }
  a.kchunk = kchunk;
  a.pstride = (size_t)nchunk * a.tiles_m * TC_M * TC_NMAX;
  const size_t smem = tc_gram_smem_bytes((q + 15) & ~15);
  tc_gram_kernel<<<dim3(nchunk, a.tiles_m, 1), TC_THREADS, smem, st>>>(b.d_elems, a, partial);
  tc_gram_reduce_kernel<<<dim3((p * q + 255) / 256, 1, 1), 256, 0, st>>>(b.d_elems, a, partial, nchunk, 2);
}

}  // namespace dgdft
