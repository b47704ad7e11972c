// Tensor-core Gram products for the FP32 stage (Sec. II.B, operation 2).
//
// C = U^T V over the N_g rows of each element, where U is a concatenation of
// up to 6 column blocks (the MMA M side, 128-row tiles) and V of up to 3
// blocks (the N side, <= 144 columns).  Every FP32 value x is split into
// bf16 parts hi = bf16(x), lo = bf16(x - hi) and the product (hi + lo)(hi + lo)
// is formed as four bf16 tcgen05.mma (kind::f16, FP32 accumulation in tensor
// memory, M = 128, K = 16 per instruction, operands in 128-byte-swizzled
// K-major shared-memory tiles).  The kernel itself is described below.
#include <cuda_bf16.h>

#include "internal.h"

namespace dgdft {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KC = 64;                    // rows (K) per stage: one 128-byte bf16 row
constexpr int TC_NMAX = 256;                 // accumulator columns (N <= 256)
constexpr int A_BYTES = TC_M * TC_KC * 2;    // one bf16 part of the A tile: 16 KB

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

// ---------------------------------------------------------------------------
// Windowed tensor-core Gram.  Accumulating a whole chunk in tensor memory
// (FP32) would limit the accuracy: the error grows with the number of
// accumulations, ~1e-5 relative over 2048 rows.  Here the
// dominant product hi*hi accumulates in tensor memory for a window of four
// 64-row steps (16 accumulations); after each window epilogue warps read it out with
// tcgen05.ld and add it to two-sum compensated registers, while the next
// window accumulates into the other of two tensor-memory buffers.  The three
// small products (hi*lo, lo*hi, lo*lo, 2^-8 and below) accumulate over the
// chunk in a third buffer.
//
// Warp roles (16 warps): warps 0-3 stage FP32 tiles with cp.async (two steps
// ahead), split them into the bf16 hi/lo swizzled tiles and (thread 0) issue
// the MMAs; warps 4-15 are the epilogue, three per tensor-memory lane quarter
// (warp w reads lanes 32 (w % 4)), 48 columns each.  Every mbarrier wait is
// bounded; on expiry the element's state records an error and the CTA stops.
constexpr int TW_KS = 64;
constexpr int TW_WIN = 4;  // 64-row steps per tensor-memory window of the hi*hi product
constexpr int TW_NMAX = 144;
constexpr int TW_PROD = 4;
constexpr int TW_EPI = 12;
constexpr int TW_THREADS = 32 * (TW_PROD + TW_EPI);
constexpr int TW_STG = (TC_M + TW_NMAX) * TW_KS * 4;  // one FP32 staging step: 68 KB

// Bounded wait that sleeps between polls, so waiting warps do not take issue
// slots from the warps doing the work; gives up after ~2^22 polls (about a
// second) and returns false.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity) {
  unsigned ns = 32;
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
  return false;
}

// Split eight consecutive k values (k0 % 8 == 0) of row r and store the hi
// and lo parts as one 16-byte chunk each of the 128B-swizzled tiles.
__device__ __forceinline__ void split_store8(unsigned char* hi, unsigned char* lo, int r, int k0, const float4& a,
                                             const float4& b) {
  const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hp = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hp);
    const __nv_bfloat162 lp = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hp);
    l[i] = *reinterpret_cast<const uint32_t*>(&lp);
  }
  const uint32_t off = sw128_off(r, k0);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void named_sync_producers() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Barrier of the 128 producer threads that also ORs a flag across them, so
// every producer takes the same branch after it.
__device__ __forceinline__ int named_sync_or_producers(int flag) {
  int r;
  asm volatile(
      "{\n"
      " .reg .pred p, q;\n"
      " setp.ne.s32 p, %1, 0;\n"
      " bar.red.or.pred q, 1, 128, p;\n"
      " selp.s32 %0, 1, 0, q;\n"
      "}\n"
      : "=r"(r)
      : "r"(flag)
      : "memory");
  return r;
}

// grid: (nchunk, tiles_m, nel); dynamic smem: tcw_gram_smem_bytes(N).
__global__ void __launch_bounds__(TW_THREADS, 1)
    tcw_gram_kernel(const ElemDev<float>* __restrict__ elems, TcGramArgs args, double* __restrict__ partial) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bar_empty, bar_dfull[2], bar_dempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ const float* colptr[TC_M + TW_NMAX];  // source column of each staged column (nullptr: zero)
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  const int M_total = args.a.nblk * side_cols(e, args.a);
  const int N_real = args.b.nblk * side_cols(e, args.b);
  const int N = (N_real + 15) & ~15;
  const int mt = blockIdx.y;
  if (mt * TC_M >= M_total || N > TW_NMAX) return;
  const int rows = e.ng;
  if (rows & 3) {
    // bulk copies need 16-byte aligned columns: the host routes such
    // elements to the other kernel; record it if one arrives here anyway
    if (threadIdx.x == 0) atomicOr(&e.state[ST_ERROR], ERR_EIG);
    return;
  }
  const int k_beg = blockIdx.x * args.kchunk;
  const int k_end = min(rows, k_beg + args.kchunk);
  const int nsteps = (k_end > k_beg) ? (k_end - k_beg + TW_KS - 1) / TW_KS : 0;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* stg0 = reinterpret_cast<float*>(base);
  float* stg1 = reinterpret_cast<float*>(base + TW_STG);
  unsigned char* a_hi = base + 2 * TW_STG;
  unsigned char* a_lo = a_hi + A_BYTES;
  const int b_bytes = ((N + 7) / 8) * 1024;
  unsigned char* b_hi = a_lo + A_BYTES;
  unsigned char* b_lo = b_hi + b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_empty, 1);
    mbar_init(&bar_dfull[0], 1);
    mbar_init(&bar_dfull[1], 1);
    mbar_init(&bar_dempty[0], TW_EPI);
    mbar_init(&bar_dempty[1], TW_EPI);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t d_rest = tmem + 2 * TW_NMAX;

  if (warp < TW_PROD) {
    // ---------------- producers: stage, split, issue ----------------
    const int ptid = tid;
    // resolve every staged column's source once (block lookups read the
    // element descriptor and its state word from global memory)
    for (int col = ptid; col < TC_M + N; col += 32 * TW_PROD) {
      const float* src = nullptr;
      if (col < TC_M) {
        const int gc = mt * TC_M + col;
        src = (gc < M_total) ? side_col(e, args.a, gc) : nullptr;
      } else {
        const int bc = col - TC_M;
        src = (bc < N_real) ? side_col(e, args.b, bc) : nullptr;
      }
      colptr[col] = src;
    }
    const float* dummy = reinterpret_cast<const float*>(e.state);
    named_sync_producers();
    // 16-byte cp.async per 4 rows of a column (rows % 4 == 0: aligned), two
    // steps ahead; sources past the chunk or without a column are zero-filled
    auto issue_loads = [&](int c, float* st) {
      const int k0 = k_beg + c * TW_KS;
      const int ncol = TC_M + N;
      for (int t = ptid; t < ncol * (TW_KS / 4); t += 32 * TW_PROD) {
        const int col = t >> 4, q = t & 15;  // TW_KS / 4 = 16 chunks per column
        const float* src = colptr[col];
        const int k = k0 + 4 * q;
        const int nv = src ? max(0, min(4, k_end - k)) : 0;
        cp_async16(st + col * TW_KS + 4 * q, nv ? src + k : dummy, 4 * nv);
      }
      cp_async_commit();
    };
    const uint32_t idesc = idesc_bf16_f32(TC_M, N);
    if (nsteps > 0) issue_loads(0, stg0);
    if (nsteps > 1) issue_loads(1, stg1);
    else cp_async_commit();
    int last_issued = -1;  // thread 0: the last step whose MMAs were issued
    for (int c = 0; c < nsteps; ++c) {
      float* st = (c & 1) ? stg1 : stg0;
      cp_async_wait<1>();  // this thread's copies of step c have landed
      bool ok = true;
      if (c >= 1) ok = mbar_wait_sleep(&bar_empty, (c - 1) & 1);  // the tile is free again
      if (named_sync_or_producers(!ok || abort_flag != 0)) {
        if (ptid == 0) atomicOr(&abort_flag, 1);
        break;
      }
      // split: a thread takes 8 consecutive k of one column (one 16-byte
      // chunk of the swizzled bf16 row); eight lanes cover a column's 64 k
      const int ncol = TC_M + N;
      for (int t = ptid; t < ncol * (TW_KS / 8); t += 32 * TW_PROD) {
        const int col = t >> 3, k8 = (t & 7) * 8;
        const float4* src = reinterpret_cast<const float4*>(st + col * TW_KS + k8);
        const float4 v0 = src[0], v1 = src[1];
        if (col < TC_M) split_store8(a_hi, a_lo, col, k8, v0, v1);
        else split_store8(b_hi, b_lo, col - TC_M, k8, v0, v1);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync_producers();
      if (c + 2 < nsteps) issue_loads(c + 2, st);
      else cp_async_commit();
      if (ptid == 0) {
        const int wi = c / TW_WIN, b = wi & 1;
        const bool first = (c % TW_WIN) == 0, last = (c % TW_WIN) == TW_WIN - 1 || c == nsteps - 1;
        bool ok = true;
        if (first && wi >= 2) ok = mbar_wait_sleep(&bar_dempty[b], ((wi >> 1) - 1) & 1);
        if (!ok) {
          atomicOr(&abort_flag, 1);
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dhh = tmem + b * TW_NMAX;
          const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
          for (int kk = 0; kk < TW_KS / 16; ++kk) {
            const uint32_t koff = kk * 32;
            mma_bf16(dhh, sw128_desc(ah + koff), sw128_desc(bh + koff), idesc, (!first || kk > 0) ? 1u : 0u);
            mma_bf16(d_rest, sw128_desc(ah + koff), sw128_desc(bl + koff), idesc, (c > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d_rest, sw128_desc(al + koff), sw128_desc(bh + koff), idesc, 1u);
            mma_bf16(d_rest, sw128_desc(al + koff), sw128_desc(bl + koff), idesc, 1u);
          }
          mma_commit(&bar_empty);
          if (last) mma_commit(&bar_dfull[b]);
          last_issued = c;
        }
      }
    }
    cp_async_wait<0>();  // no copy may land after the CTA exits
    // the last issued MMAs must finish before tensor memory is released
    if (ptid == 0 && last_issued >= 0) {
      if (!mbar_wait_sleep(&bar_empty, last_issued & 1)) atomicOr(&abort_flag, 1);
    }
  } else {
    // ---------------- epilogue: windowed read-out ----------------
    const int ew = warp - TW_PROD;
    const int quarter = warp & 3, g = ew >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    float hi[48], lo[48];
#pragma unroll
    for (int j = 0; j < 48; ++j) hi[j] = lo[j] = 0.f;
    const int nwin = (nsteps + TW_WIN - 1) / TW_WIN;
    for (int wi = 0; wi < nwin; ++wi) {
      const int b = wi & 1;
      if (!mbar_wait_sleep(&bar_dfull[b], (wi >> 1) & 1)) {
        atomicOr(&abort_flag, 1);
        break;
      }
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float v[16];
        tmem_ld16(tmem + lane_base + (uint32_t)(b * TW_NMAX + 48 * g + 16 * i), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float x = v[j], h = hi[16 * i + j];
          const float sum = h + x;
          const float bp = sum - h;
          lo[16 * i + j] += (h - (sum - bp)) + (x - bp);
          hi[16 * i + j] = sum;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_dempty[b]);
    }
    if (!abort_flag && nsteps > 0) {
      // the last dfull completion covers every MMA, the small products included
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      double* out = partial + blockIdx.z * args.pstride +
                    ((size_t)blockIdx.x * args.tiles_m + mt) * ((size_t)TC_M * TC_NMAX);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float v[16];
        tmem_ld16(d_rest + lane_base + (uint32_t)(48 * g + 16 * i), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = 48 * g + 16 * i + j;
          if (col < N) out[(size_t)row * TC_NMAX + col] = (double)hi[16 * i + j] + (double)lo[16 * i + j] +
                                                           (double)v[j];
        }
      }
    } else if (nsteps == 0) {
      double* out = partial + blockIdx.z * args.pstride +
                    ((size_t)blockIdx.x * args.tiles_m + mt) * ((size_t)TC_M * TC_NMAX);
      for (int j = 0; j < 48; ++j)
        if (48 * g + j < N) out[(size_t)row * TC_NMAX + 48 * g + j] = 0.0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_flag) atomicOr(&e.state[ST_ERROR], ERR_EIG);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
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

size_t tcw_gram_smem_bytes(int n_cols) {
  const int b_bytes = ((n_cols + 7) / 8) * 1024;
  return 2 * (size_t)TW_STG + 2 * (size_t)A_BYTES + 2 * (size_t)b_bytes + 1024;
}

void init_tc_gram_kernel() { opt_in_dynamic_smem((const void*)tcw_gram_kernel); }

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
  const int n16 = ((a.b.nblk * m) + 15) & ~15;
  tcw_gram_kernel<<<dim3(nchunk, a.tiles_m, b.s.nel), TW_THREADS, tcw_gram_smem_bytes(n16), st>>>(b.d_elems, a,
                                                                                                partial);
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
  const int q16 = (q + 15) & ~15;
  tcw_gram_kernel<<<dim3(nchunk, a.tiles_m, 1), TW_THREADS, tcw_gram_smem_bytes(q16), st>>>(b.d_elems, a, partial);
  tc_gram_reduce_kernel<<<dim3((p * q + 255) / 256, 1, 1), 256, 0, st>>>(b.d_elems, a, partial, nchunk, 2);
}

}  // namespace dgdft
