// Tensor-core Gram products of the FP32 stage (Sec. II.B, operation 2: the 12
// products Phi^T Psi of an iteration, and X^T W for the projection of W).
//
// Precision.  Every FP32 value x is split into two TF32 values,
// hi = rn_tf32(x) and lo = rn_tf32(x - hi), so that hi + lo = x (1 + d) with
// |d| <= 2^-22; a product is formed as hi*hi + hi*lo + lo*hi by three
// tcgen05.mma kind::tf32 instructions (the dropped lo*lo is below 2^-22 of
// the product).  The tensor core accumulates in FP32 in tensor memory for a
// window of 256 rows; after each window the epilogue warps add the window
// sums into two-sum compensated FP32 registers, and a CTA's chunk total goes
// as the (hi, lo) pair to a partial buffer that is reduced in a fixed order
// in FP64.
//
// Data movement.  The blocks are column-major N_g x m FP32 (m <= 48), so a
// vector's grid rows are contiguous: both MMA operands are K-major with the
// grid rows as K.  A stage is 32 grid rows of four blocks; each block is
// loaded by one TMA copy (box 32 rows x 48 columns, 128-byte swizzle) into a
// 48-row slot of 128-byte rows, which is the canonical K-major SW128 layout
// the MMA reads.  Columns beyond m and rows beyond N_g are filled with zeros
// by the copy.  The split warps overwrite a slot with hi in place and write
// lo to a second buffer of the same layout.
//
// Which products.  With S = [X W P], the Rayleigh-Ritz pencil needs the
// upper block triangles of A = (H S)^T S and B = S^T S: 12 blocks of m x m.
// They are covered by two CTA types (M = 128 rows of the accumulator):
//   type 0: slots [HX X W P]; D = rows 0..127 ([HX X W(0:32)]) times rows
//           48..191 ([X W P], N = 144);
//   type 1: slots [HP P W HW]; D1 = rows 64..191 ([P(16:48) W HW]) times
//           rows 48..143 ([P W], N = 96), D2 = rows 0..127 ([HP P W(0:32)])
//           times rows 48..95 (P, N = 48);
// 3/4 of the MMA area is used.  X^T W (mode 1) is type 2: slots [W X],
// D = rows 0..127 times rows 48..95 (X, N = 48).
//
// Scheduling.  A persistent grid of one CTA per SM.  Every CTA lists the
// active elements from their state words (the list is the same in every
// CTA); each (element, type) is split into C row chunks with C chosen from
// the grid size and the active count, and CTA b takes items b, b + G, ...
// Warp roles: warp 0 issues the TMA copies, warp 1 the MMAs, warps 2-3
// split, warps 4-15 read tensor memory (three warps per lane quarter, 48
// accumulator columns each).  Every mbarrier wait is bounded; on expiry the
// element records ERR_TIMEOUT, the CTA waits (with the default limit) for its
// copies and MMAs in flight, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "tcgen05.cuh"

namespace dgdft {

namespace {

constexpr int SLOT = 48;                         // rows (block columns) per slot
constexpr int NSLOT = 4;                         // slots per stage
constexpr int KS = 32;                           // grid rows per stage
constexpr int ROWB = KS * 4;                     // bytes per staged column: one 128-byte swizzle row
constexpr int SLOT_BYTES = SLOT * ROWB;          // 6144
constexpr int STAGE_BYTES = NSLOT * SLOT_BYTES;  // 24576 for hi, as much again for lo
constexpr int NST = 4;                           // pipeline depth (stages in shared memory)
constexpr int WIN = 8;                           // stages per tensor-memory window (256 rows)
constexpr int MT = 128;                          // MMA M
constexpr int NACC = 144;                        // accumulator columns per window buffer
constexpr int NEPI = 12;                         // epilogue warps
constexpr int THREADS = 32 * (4 + NEPI);         // 512
constexpr int PART = MT * NACC;                  // (hi, lo) pairs per partial (one item)
constexpr int MAX_SCHED_EL = 1024;               // elements a launch can schedule
constexpr size_t DYN_SMEM = 2 * (size_t)NST * STAGE_BYTES + 1024;
constexpr uint32_t DEFAULT_POLLS = 1u << 22;     // blocking tests: 0.1 s to a few s

struct MmaOp {
  int a_row, b_row, n, d_col;
};
struct Recipe {
  int nslot;
  int sel[NSLOT];
  int nmma;
  MmaOp mma[2];
};

__device__ __forceinline__ Recipe recipe(int type) {
  Recipe r{};
  if (type == 0) {
    r.nslot = 4;
    r.sel[0] = BHX; r.sel[1] = BX; r.sel[2] = BW; r.sel[3] = BP;
    r.nmma = 1;
    r.mma[0] = MmaOp{0, 48, 144, 0};
  } else if (type == 1) {
    r.nslot = 4;
    r.sel[0] = BHP; r.sel[1] = BP; r.sel[2] = BW; r.sel[3] = BHW;
    r.nmma = 2;
    r.mma[0] = MmaOp{64, 48, 96, 0};
    r.mma[1] = MmaOp{0, 48, 48, 96};
  } else {
    r.nslot = 2;
    r.sel[0] = BW; r.sel[1] = BX;
    r.nmma = 1;
    r.mma[0] = MmaOp{0, 48, 48, 0};
  }
  return r;
}

// Tensor map of block `sel` of element `e` (10 per element: X, P, HX, HP in
// both buffers, then W, HW).
__device__ __forceinline__ const void* block_map(const unsigned char* maps, int e, int sel, int parity) {
  const int idx = sel < NDBL ? sel * 2 + parity : 2 * NDBL + (sel - NDBL);
  return maps + ((size_t)e * 10 + idx) * 128;
}

struct Sched {
  int nact, ntypes, C, total;
};

// Items of the launch: (active element a, type t, chunk c), a-major.
__device__ __forceinline__ Sched make_sched(int nact, int ntypes, int G, int cmax) {
  Sched s;
  s.nact = nact;
  s.ntypes = ntypes;
  int C = nact > 0 ? G / (nact * ntypes) : 1;
  C = C < 1 ? 1 : (C > cmax ? cmax : C);
  s.C = C;
  s.total = nact * ntypes * C;
  return s;
}

struct Item {
  int e, type, chunk, r0, nst;
};

__device__ __forceinline__ Item decode(int i, const Sched& s, const int* act, int mode,
                                       const ElemDev<float>* elems) {
  Item it;
  const int per = s.ntypes * s.C;
  const int a = i / per, rem = i - a * per;
  it.e = act[a];
  it.type = mode == 0 ? rem / s.C : 2;
  it.chunk = rem % s.C;
  const int ng = elems[it.e].ng;
  const int R = (((ng + s.C - 1) / s.C) + KS - 1) / KS * KS;
  it.r0 = it.chunk * R;
  const int r1 = min(ng, it.r0 + R);
  it.nst = r1 > it.r0 ? (r1 - it.r0 + KS - 1) / KS : 0;
  return it;
}

__global__ void __launch_bounds__(THREADS, 1)
    tf32_gram_kernel(const ElemDev<float>* __restrict__ elems, int nel, const unsigned char* __restrict__ maps,
                     int mode, int cmax, uint32_t polls, double* __restrict__ partial) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bar_full[NST], bar_conv[NST], bar_empty[NST], bar_dfull[2], bar_dempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int act[MAX_SCHED_EL];
  __shared__ int nact_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* hi_buf = base;                           // NST stages of STAGE_BYTES
  unsigned char* lo_buf = base + (size_t)NST * STAGE_BYTES;
  if (tid == 0) {
    int n = 0;
    for (int e = 0; e < nel && e < MAX_SCHED_EL; ++e)
      if (elems[e].state[ST_ACTIVE]) act[n++] = e;
    nact_s = n;
    abort_flag = 0;
    for (int s = 0; s < NST; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_conv[s], 2);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_dfull[b], 1);
      mbar_init(&bar_dempty[b], NEPI);
    }
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
  const int ntypes = mode == 0 ? 2 : 1;
  const Sched sc = make_sched(nact_s, ntypes, (int)gridDim.x, cmax);
  const uint32_t cleanup_polls = DEFAULT_POLLS;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t stage = 0;
      for (int i = blockIdx.x; i < sc.total && !abort_flag; i += gridDim.x) {
        const Item it = decode(i, sc, act, mode, elems);
        const Recipe rc = recipe(it.type);
        const int par = elems[it.e].state[ST_PARITY] & 1;
        for (int j = 0; j < it.nst; ++j, ++stage) {
          const int s = stage % NST;
          if (stage >= NST && !mbar_wait(&bar_empty[s], ((stage / NST) - 1) & 1, polls)) {
            atomicOr(&elems[it.e].state[ST_ERROR], ERR_TIMEOUT);
            atomicOr(&abort_flag, 1);
            break;
          }
          if (abort_flag) break;
          mbar_expect_tx(&bar_full[s], (uint32_t)(rc.nslot * SLOT_BYTES));
#pragma unroll
          for (int q = 0; q < NSLOT; ++q)
            if (q < rc.nslot)
              tma_load(hi_buf + (size_t)s * STAGE_BYTES + q * SLOT_BYTES, block_map(maps, it.e, rc.sel[q], par),
                       it.r0 + j * KS, 0, &bar_full[s]);
        }
      }
      // no copy may land after the CTA exits: wait for the last issued
      // copy of every stage slot (their phases complete in issue order)
      for (uint32_t k = 0; k < NST && k < stage; ++k) {
        const uint32_t st = stage - 1 - k;
        mbar_wait(&bar_full[st % NST], (st / NST) & 1, cleanup_polls);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, win = 0;
      bool issued = false;
      uint32_t last_stage = 0;
      for (int i = blockIdx.x; i < sc.total && !abort_flag; i += gridDim.x) {
        const Item it = decode(i, sc, act, mode, elems);
        const Recipe rc = recipe(it.type);
        for (int j = 0; j < it.nst; ++j, ++stage) {
          const int s = stage % NST;
          const bool first = (j % WIN) == 0, last = (j % WIN) == WIN - 1 || j == it.nst - 1;
          const uint32_t b = win & 1;
          bool ok = mbar_wait(&bar_conv[s], (stage / NST) & 1, polls);
          if (ok && first && win >= 2) ok = mbar_wait(&bar_dempty[b], ((win >> 1) - 1) & 1, polls);
          if (!ok) {
            atomicOr(&elems[it.e].state[ST_ERROR], ERR_TIMEOUT);
            atomicOr(&abort_flag, 1);
            break;
          }
          if (abort_flag) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t hs = smem_u32(hi_buf + (size_t)s * STAGE_BYTES);
          const uint32_t ls = smem_u32(lo_buf + (size_t)s * STAGE_BYTES);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            if (q >= rc.nmma) break;
            const MmaOp op = rc.mma[q];
            const uint32_t idesc = idesc_tf32(MT, op.n);
            const uint32_t d = tmem + b * NACC + op.d_col;
#pragma unroll
            for (int kk = 0; kk < KS / 8; ++kk) {
              const uint32_t ko = kk * 32;
              const uint64_t ah = sw128_desc(hs + op.a_row * ROWB + ko), bh = sw128_desc(hs + op.b_row * ROWB + ko);
              const uint64_t al = sw128_desc(ls + op.a_row * ROWB + ko), bl = sw128_desc(ls + op.b_row * ROWB + ko);
              mma_tf32(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
              mma_tf32(d, ah, bl, idesc, 1u);
              mma_tf32(d, al, bh, idesc, 1u);
            }
          }
          mma_commit(&bar_empty[s]);
          issued = true;
          last_stage = stage;
          if (last) {
            mma_commit(&bar_dfull[b]);
            ++win;
          }
        }
      }
      // the MMAs must finish before tensor memory is released
      if (issued) mbar_wait(&bar_empty[last_stage % NST], (last_stage / NST) & 1, cleanup_polls);
    }
  } else if (warp < 4) {
    // ------------------------------------------------ split into hi / lo
    const int ct = tid - 64;  // 0..63
    uint32_t stage = 0;
    for (int i = blockIdx.x; i < sc.total && !abort_flag; i += gridDim.x) {
      const Item it = decode(i, sc, act, mode, elems);
      const int nvec = recipe(it.type).nslot * SLOT_BYTES / 16;
      for (int j = 0; j < it.nst; ++j, ++stage) {
        const int s = stage % NST;
        if (!mbar_wait(&bar_full[s], (stage / NST) & 1, polls)) {
          atomicOr(&elems[it.e].state[ST_ERROR], ERR_TIMEOUT);
          atomicOr(&abort_flag, 1);
          break;
        }
        if (abort_flag) break;
        float4* h4 = reinterpret_cast<float4*>(hi_buf + (size_t)s * STAGE_BYTES);
        float4* l4 = reinterpret_cast<float4*>(lo_buf + (size_t)s * STAGE_BYTES);
#pragma unroll 4
        for (int t = ct; t < nvec; t += 64) {
          const float4 x = h4[t];
          float4 h, l;
          h.x = rn_tf32(x.x); l.x = rn_tf32(x.x - h.x);
          h.y = rn_tf32(x.y); l.y = rn_tf32(x.y - h.y);
          h.z = rn_tf32(x.z); l.z = rn_tf32(x.z - h.z);
          h.w = rn_tf32(x.w); l.w = rn_tf32(x.w - h.w);
          h4[t] = h;
          l4[t] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_conv[s]);
      }
    }
  } else {
    // ------------------------------------------------ epilogue
    const int ew = warp - 4;
    const int quarter = warp & 3, g = ew >> 2;  // lane quarter, column group
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    uint32_t win = 0;
    for (int i = blockIdx.x; i < sc.total; i += gridDim.x) {
      const Item it = decode(i, sc, act, mode, elems);
      float hi[48], lo[48];
#pragma unroll
      for (int j = 0; j < 48; ++j) hi[j] = lo[j] = 0.f;
      const int nwin = (it.nst + WIN - 1) / WIN;
      const int slot = (it.e * ntypes + (mode == 0 ? it.type : 0)) * cmax + it.chunk;
      float2* out2 = reinterpret_cast<float2*>(partial) + (size_t)slot * PART;
      bool ok = !abort_flag;
      for (int w = 0; w < nwin && ok; ++w, ++win) {
        const uint32_t b = win & 1;
        if (!mbar_wait(&bar_dfull[b], (win >> 1) & 1, polls)) {
          atomicOr(&elems[it.e].state[ST_ERROR], ERR_TIMEOUT);
          atomicOr(&abort_flag, 1);
          ok = false;
          break;
        }
        if (abort_flag) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool final_win = w == nwin - 1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float v[16];
          tmem_ld16(tmem + lane_base + (uint32_t)(b * NACC + 48 * g + 16 * q), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float x = v[j], h = hi[16 * q + j];
            const float sum = h + x;
            const float bp = sum - h;
            lo[16 * q + j] += (h - (sum - bp)) + (x - bp);
            hi[16 * q + j] = sum;
          }
          if (final_win) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              out2[(size_t)(48 * g + 16 * q + j) * MT + row] = make_float2(hi[16 * q + j], lo[16 * q + j]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_dempty[b]);
      }
      if (!ok) break;
      if (nwin == 0)
        for (int j = 0; j < 48; ++j) out2[(size_t)(48 * g + j) * MT + row] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Where output (block q, r, c) of the LOBPCG pencil was accumulated: the
// item type and the accumulator row and column (see the recipes).  Blocks
// 0-5 are A = (H S)^T S: (HX,X) (HX,W) (HX,P) (HW,W) (HW,P) (HP,P); blocks
// 6-11 are B = S^T S: (X,X) (X,W) (X,P) (W,W) (W,P) (P,P).
__device__ __forceinline__ void source_of(int q, int r, int c, int& type, int& drow, int& dcol) {
  switch (q) {
    case 0: type = 0; drow = r; dcol = c; break;
    case 1: type = 0; drow = r; dcol = 48 + c; break;
    case 2: type = 0; drow = r; dcol = 96 + c; break;
    case 3: type = 1; drow = 80 + r; dcol = 48 + c; break;
    case 4: type = 1; drow = 80 + r; dcol = c; break;
    case 5: type = 1; drow = r; dcol = 96 + c; break;
    case 6: type = 0; drow = 48 + r; dcol = c; break;
    case 7: type = 0; drow = 48 + r; dcol = 48 + c; break;
    case 8: type = 0; drow = 48 + r; dcol = 96 + c; break;
    case 9:
      if (r < 32) { type = 0; drow = 96 + r; dcol = 48 + c; }
      else { type = 1; drow = 32 + r; dcol = 48 + c; }
      break;
    case 10:
      if (r < 32) { type = 0; drow = 96 + r; dcol = 96 + c; }
      else { type = 1; drow = 32 + r; dcol = c; }
      break;
    default:
      if (r >= 16) { type = 1; drow = r - 16; dcol = c; }
      else { type = 1; drow = 48 + r; dcol = 96 + c; }
      break;
  }
}

// Sums the chunk partials of every element in a fixed order and writes the
// Gram blocks: mode 0 the upper block triangles of A and B (ld 3m), mode 1
// X^T W (gxw, ld m).  The active count is read as the Gram kernel read it
// (nothing changes the state words in between), so both derive the same C.
__global__ void tf32_gram_reduce_kernel(const ElemDev<float>* __restrict__ elems, int nel, int mode, int G,
                                        int cmax, const double* __restrict__ partial) {
  const ElemDev<float>& e = elems[blockIdx.z];
  if (!e.state[ST_ACTIVE]) return;
  __shared__ int nact;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int k = 0; k < nel && k < MAX_SCHED_EL; ++k) n += elems[k].state[ST_ACTIVE] != 0;
    nact = n;
  }
  __syncthreads();
  const int ntypes = mode == 0 ? 2 : 1;
  const Sched sc = make_sched(nact, ntypes, G, cmax);
  // a timed-out element keeps its stale Gram; the Rayleigh-Ritz step stops it
  if (e.state[ST_ERROR] & ERR_TIMEOUT) return;
  const int m = e.m;
  const bool has_p = e.state[ST_HAS_P] != 0;
  const float2* part2 = reinterpret_cast<const float2*>(partial);
  const int nout = (mode == 0 ? 12 : 1) * m * m;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nout; idx += gridDim.x * blockDim.x) {
    const int q = idx / (m * m), rc = idx - q * m * m;
    const int r = rc / m, c = rc - r * m;
    int type = 2, drow = r, dcol = c;
    if (mode == 0) source_of(q, r, c, type, drow, dcol);
    const int ti = mode == 0 ? type : 0;
    double s = 0.0;
    const bool zero = mode == 0 && !has_p && (q == 2 || q == 4 || q == 5 || q == 8 || q == 10 || q == 11);
    if (!zero)
      for (int ch = 0; ch < sc.C; ++ch) {
        const float2 v = part2[((size_t)(blockIdx.z * ntypes + ti) * cmax + ch) * PART + (size_t)dcol * MT + drow];
        s += (double)v.x + (double)v.y;
      }
    if (mode == 0) {
      const int bi = q < 6 ? (q < 3 ? 0 : (q < 5 ? 1 : 2)) : (q < 9 ? 0 : (q < 11 ? 1 : 2));
      const int qq = q % 6;
      const int bj = qq == 0 ? 0 : (qq == 1 || qq == 3) ? 1 : 2;
      double* out = e.gram + (q < 6 ? 0 : (size_t)9 * m * m);
      out[(bi * m + r) + (size_t)(bj * m + c) * (3 * m)] = s;
    } else {
      e.gxw[c + (size_t)r * m] = s;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
int g_num_sms = 0;

}  // namespace

bool tf32_gram_eligible(const BatchShape& s) {
  return s.max_m <= SLOT && s.ng_mult4 && s.nel <= MAX_SCHED_EL && s.nel > 0;
}

size_t tf32_gram_partial_doubles(int nel, int cmax) { return (size_t)nel * 2 * cmax * PART; }

std::string encode_tf32_gram_maps(const ElemDev<float>* h, int nel, void* host_out) {
  std::call_once(g_encode_once, []() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return "cuTensorMapEncodeTiled is not available";
  unsigned char* out = static_cast<unsigned char*>(host_out);
  for (int e = 0; e < nel; ++e) {
    for (int idx = 0; idx < 10; ++idx) {
      const int sel = idx < 2 * NDBL ? idx / 2 : NDBL + (idx - 2 * NDBL);
      const int buf = idx < 2 * NDBL ? (idx & 1) : 0;
      void* ptr = h[e].blk[sel][buf];
      if (((uintptr_t)ptr & 15) || (h[e].ng & 3)) return "block not 16-byte aligned";
      cuuint64_t dims[2] = {(cuuint64_t)h[e].ng, (cuuint64_t)h[e].m};
      cuuint64_t strides[1] = {(cuuint64_t)h[e].ng * 4};
      cuuint32_t box[2] = {(cuuint32_t)KS, (cuuint32_t)SLOT};
      cuuint32_t estr[2] = {1, 1};
      CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out + ((size_t)e * 10 + idx) * 128);
      const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    }
  }
  return "";
}

void init_tf32_gram_kernel() {
  cudaFuncSetAttribute((const void*)tf32_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DYN_SMEM);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
}

bool launch_tf32_gram(const Batch<float>& b, const void* d_maps, int mode, double* partial, size_t partial_cap,
                      uint32_t polls, cudaStream_t st) {
  const int nel = b.s.nel;
  const int ntypes = mode == 0 ? 2 : 1;
  const int cmax = (int)std::min<size_t>(32, partial_cap / ((size_t)nel * ntypes * PART));
  if (cmax < 1 || !tf32_gram_eligible(b.s)) return false;
  const int G = g_num_sms > 0 ? g_num_sms : 148;
  const uint32_t p = polls ? polls : DEFAULT_POLLS;
  tf32_gram_kernel<<<G, THREADS, DYN_SMEM, st>>>(b.d_elems, nel, static_cast<const unsigned char*>(d_maps), mode,
                                                 cmax, p, partial);
  const int nout = (mode == 0 ? 12 : 1) * b.s.max_m * b.s.max_m;
  tf32_gram_reduce_kernel<<<dim3((nout + 255) / 256, 1, nel), 256, 0, st>>>(b.d_elems, nel, mode, G, cmax,
                                                                           partial);
  return true;
}

}  // namespace dgdft
