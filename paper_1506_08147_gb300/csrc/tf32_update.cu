// Tensor-core block updates of the FP32 stage (Sec. II.B, operation 4: the
// paper's Phi C products).
//
// out = alpha sum_i in_i Y_i + beta out, and optionally out2 = the sum over
// inputs i >= from2 of in_i Y_i, for every element of a batch: the FP32
// stage's X' = [X W P] Y (with P' = [W P] Y_wp on the way), HP' = [HW HP] Y_wp
// and the projection W - X (X^T W).  Blocks are column-major N_g x m FP32
// (m <= 48); Y is the Rayleigh-Ritz result's FP32 copy, or X^T W in FP64.
//
// Precision.  As in the tensor-core Gram (tf32_gram.cu), both operands are
// split into TF32 parts hi + lo (hi + lo = x (1 + d), |d| <= 2^-22) and a
// product is hi*hi + hi*lo + lo*hi, three tcgen05.mma kind::tf32 per K step.
// A sum runs over at most 3m = 144 terms, accumulated in FP32 in tensor
// memory.
//
// Shape.  D = 128 grid rows (the MMA's M) x N output columns (m rounded up to
// 16).  K runs over the active inputs' columns, each input padded to Kin (m
// rounded up to 16) and packed in 32-column chunks, one 128-byte row of the
// K-major, 128-byte-swizzled operand layout; inputs are packed last first, as
// the SIMT kernel sums them.  An 8-wide K step lies inside one input and
// accumulates into D0 (inputs before from2) or D1 (inputs from from2 on), so
// out and out2 come out of one pass.
//
// Roles (persistent grid, one CTA per SM; the items (element, 128-row tile)
// are ordered by element and split into one contiguous range per CTA):
// warp 0 issues TMA copies of 128 rows x 16 columns of an input (unswizzled,
// rows contiguous) into a ring of chunk stages; warps 2-5 transpose each
// staged chunk into the K-major layout as hi and lo parts, and split Y into
// the B operand when the element changes (after the MMAs of the previous
// element have completed); warp 1 issues the MMAs into one of two
// accumulator pairs in tensor memory; warps 6-9 read the accumulators (one
// lane quarter each) and write out and out2 with coalesced stores.  Every
// mbarrier wait is bounded; on expiry the element records ERR_TIMEOUT, the
// CTA waits (with the default limit) for its copies and MMAs in flight, frees
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "tcgen05.cuh"

namespace dgdft {

namespace {

constexpr int UM = 128;                               // grid rows per tile (MMA M)
constexpr int UKC = 32;                               // packed K per chunk
constexpr int UNMAX = 48;                             // output columns at most
constexpr int UNCH = 5;                               // chunks at most: 3 x 48 = 144 -> 5 x 32
constexpr int UNST = 3;                               // chunk stages in flight
constexpr int UBOX = 16;                              // columns per TMA copy
constexpr size_t STG_BYTES = (size_t)UKC * UM * 4;    // FP32 staging of a chunk: 16 KB
constexpr size_t OPA_BYTES = (size_t)UM * 128;        // A operand of a chunk (128 rows x 128 B): 16 KB
constexpr size_t STAGE_BYTES_U = STG_BYTES + 2 * OPA_BYTES;
constexpr size_t OPB_CHUNK = (size_t)UNMAX * 128;     // B operand of a chunk: 6 KB
constexpr size_t OPB_BYTES = UNCH * OPB_CHUNK;        // 30 KB for hi, as much for lo
constexpr size_t UDYN_SMEM = 2 * OPB_BYTES + UNST * STAGE_BYTES_U + 1024;
constexpr int NSPLIT = 4;                             // transpose/split warps
constexpr int NEPI_U = 4;                             // epilogue warps
constexpr int UTHREADS = 32 * (2 + NSPLIT + NEPI_U);  // 320
constexpr uint32_t UACC = 128;                        // tensor-memory columns per accumulator pair
constexpr int MAX_UPD_EL = 1024;
constexpr uint32_t UDEFAULT_POLLS = 1u << 22;

struct UpdJob {
  int nin;
  int sel[3], next[3], needs_p[3], yrow[3];
  int y_id;
  const double* y_ptr;
  int ldy;
  int out_sel, out_next, out2_sel, out2_next, from2;
  float alpha, beta;
};

// What a role needs to know about the element of an item.
struct UElem {
  int e, m, N, Kin, nai, K, nch, par;
  int in_of[3];  // packed input index -> job input
  bool has0, has1;
};

__device__ __forceinline__ UElem uelem(const ElemDev<float>* elems, const int* act, int a, const UpdJob& j) {
  UElem u;
  u.e = act[a];
  const ElemDev<float>& E = elems[u.e];
  u.m = E.m;
  u.N = (u.m + 15) & ~15;
  u.Kin = u.N;
  const bool has_p = E.state[ST_HAS_P] != 0;
  u.nai = 0;
  u.has0 = u.has1 = false;
  for (int in = j.nin - 1; in >= 0; --in) {
    if (j.needs_p[in] && !has_p) continue;
    u.in_of[u.nai++] = in;
    if (j.from2 >= 0 && in >= j.from2) u.has1 = true;
    else u.has0 = true;
  }
  u.K = u.nai * u.Kin;
  u.nch = (u.K + UKC - 1) / UKC;
  u.par = E.state[ST_PARITY] & 1;
  return u;
}

__device__ __forceinline__ int tiles_of(const ElemDev<float>& E) { return (E.ng + UM - 1) / UM; }

// Tensor map of (block sel, current or next buffer) of element e: 10 per
// element, in the order X, P, HX, HP (both buffers), W, HW.
__device__ __forceinline__ const void* umap(const unsigned char* maps, int e, int sel, int buf) {
  const int idx = sel < NDBL ? sel * 2 + buf : 2 * NDBL + (sel - NDBL);
  return maps + ((size_t)e * 10 + idx) * 128;
}

// Byte offset of (row r, packed column kc < 32) in a K-major 128-byte-swizzle
// tile: 8-row groups of 1 KB, 16-byte chunk index XOR the row within the group.
__device__ __forceinline__ uint32_t sw_off(int r, int kc) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kc >> 2) ^ r) & 7) << 4) + (kc & 3) * 4);
}

__device__ __forceinline__ float4 tf32_hi4(float4 x) {
  return make_float4(rn_tf32(x.x), rn_tf32(x.y), rn_tf32(x.z), rn_tf32(x.w));
}
__device__ __forceinline__ float4 tf32_lo4(float4 x, float4 h) {
  return make_float4(rn_tf32(x.x - h.x), rn_tf32(x.y - h.y), rn_tf32(x.z - h.z), rn_tf32(x.w - h.w));
}

// Coefficient (packed row k, output column c) of the element's Y.
__device__ __forceinline__ float ycoef(const ElemDev<float>& E, const UElem& u, const UpdJob& j, int k, int c) {
  const int ai = k / u.Kin, kl = k - ai * u.Kin;
  if (ai >= u.nai || kl >= u.m || c >= u.m) return 0.0f;
  const int row = j.yrow[u.in_of[ai]] * u.m + kl;
  if (j.y_id == Y_RR) {
    const int ldy = j.ldy > 0 ? j.ldy : 3 * u.m;
    return E.Yf[row + (size_t)c * ldy];
  }
  const double* Y = j.y_id == Y_GXW ? E.gxw : j.y_ptr;
  const int ldy = j.ldy > 0 ? j.ldy : u.m;
  return (float)Y[row + (size_t)c * ldy];
}

__global__ void __launch_bounds__(UTHREADS, 1)
    tf32_update_kernel(const ElemDev<float>* __restrict__ elems, int nel, const unsigned char* __restrict__ maps,
                       UpdJob job, uint32_t polls) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bar_full[UNST], bar_conv[UNST], bar_empty[UNST], bar_dfull[2], bar_dempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int act[MAX_UPD_EL];
  __shared__ int tile0[MAX_UPD_EL + 1];
  __shared__ int nact_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ybh = base;
  unsigned char* ybl = base + OPB_BYTES;
  unsigned char* stages = base + 2 * OPB_BYTES;
  if (tid == 0) {
    int n = 0;
    tile0[0] = 0;
    for (int e = 0; e < nel && e < MAX_UPD_EL; ++e)
      if (elems[e].state[ST_ACTIVE]) {
        act[n] = e;
        tile0[n + 1] = tile0[n] + tiles_of(elems[e]);
        ++n;
      }
    nact_s = n;
    abort_flag = 0;
    for (int s = 0; s < UNST; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_conv[s], NSPLIT);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_dfull[b], 1);
      mbar_init(&bar_dempty[b], NEPI_U);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nact = nact_s;
  const int total = tile0[nact];
  const int i0 = (int)(((long long)blockIdx.x * total) / gridDim.x);
  const int i1 = (int)(((long long)(blockIdx.x + 1) * total) / gridDim.x);
  // the element index a of item i0
  int a0 = 0;
  while (a0 < nact && tile0[a0 + 1] <= i0) ++a0;
  const uint32_t cleanup_polls = UDEFAULT_POLLS;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t stage = 0;
      int a = a0;
      UElem u{};
      if (i0 < i1) u = uelem(elems, act, a, job);  // i0 < i1: a < nact
      for (int i = i0; i < i1 && !abort_flag; ++i) {
        while (tile0[a + 1] <= i) u = uelem(elems, act, ++a, job);
        const int r0 = (i - tile0[a]) * UM;
        bool stop = false;
        for (int j = 0; j < u.nch; ++j, ++stage) {
          const int s = stage % UNST;
          if (stage >= UNST && !mbar_wait(&bar_empty[s], ((stage / UNST) - 1) & 1, polls)) {
            atomicOr(&elems[u.e].state[ST_ERROR], ERR_TIMEOUT);
            atomicOr(&abort_flag, 1);
            stop = true;
            break;
          }
          if (abort_flag) {
            stop = true;
            break;
          }
          const int nbox = (UKC * j + UBOX < u.K) ? 2 : 1;
          mbar_expect_tx(&bar_full[s], (uint32_t)(nbox * UBOX * UM * 4));
          unsigned char* stg = stages + (size_t)s * STAGE_BYTES_U;
          for (int b = 0; b < nbox; ++b) {
            const int p = UKC * j + UBOX * b;
            const int ai = p / u.Kin;
            const int in = u.in_of[ai];
            const void* map = umap(maps, u.e, job.sel[in], job.sel[in] < NDBL ? (u.par ^ job.next[in]) : 0);
            tma_load(stg + (size_t)b * UBOX * UM * 4, map, r0, p - ai * u.Kin, &bar_full[s]);
          }
        }
        if (stop) break;
      }
      // no copy may land after the CTA exits
      for (uint32_t k = 0; k < UNST && k < stage; ++k) {
        const uint32_t st = stage - 1 - k;
        mbar_wait(&bar_full[st % UNST], (st / UNST) & 1, cleanup_polls);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, win = 0, last_stage = 0;
      bool issued = false;
      int a = a0;
      UElem u{};
      if (i0 < i1) u = uelem(elems, act, a, job);  // i0 < i1: a < nact
      for (int i = i0; i < i1 && !abort_flag; ++i) {
        while (tile0[a + 1] <= i) u = uelem(elems, act, ++a, job);
        const uint32_t b = win & 1;
        bool ok = true;
        if (win >= 2) ok = mbar_wait(&bar_dempty[b], ((win >> 1) - 1) & 1, polls);
        const uint32_t idesc = idesc_tf32(UM, u.N);
        bool started[2] = {false, false};
        for (int j = 0; j < u.nch && ok; ++j, ++stage) {
          const int s = stage % UNST;
          ok = mbar_wait(&bar_conv[s], (stage / UNST) & 1, polls);
          if (!ok || abort_flag) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* stg = stages + (size_t)s * STAGE_BYTES_U;
          const uint32_t ah = smem_u32(stg + STG_BYTES), al = smem_u32(stg + STG_BYTES + OPA_BYTES);
          const uint32_t bh = smem_u32(ybh + (size_t)j * OPB_CHUNK), bl = smem_u32(ybl + (size_t)j * OPB_CHUNK);
#pragma unroll
          for (int kk = 0; kk < UKC / 8; ++kk) {
            const int ks = UKC * j + 8 * kk;
            if (ks >= u.K) break;
            const int in = u.in_of[ks / u.Kin];
            const int acc = (job.from2 >= 0 && in >= job.from2) ? 1 : 0;
            const uint32_t d = tmem + b * UACC + (uint32_t)(acc * 64);
            const uint32_t ko = (uint32_t)kk * 32;
            const uint64_t dah = sw128_desc(ah + ko), dal = sw128_desc(al + ko);
            const uint64_t dbh = sw128_desc(bh + ko), dbl = sw128_desc(bl + ko);
            mma_tf32(d, dah, dbh, idesc, started[acc] ? 1u : 0u);
            mma_tf32(d, dah, dbl, idesc, 1u);
            mma_tf32(d, dal, dbh, idesc, 1u);
            started[acc] = true;
          }
          mma_commit(&bar_empty[s]);
          issued = true;
          last_stage = stage;
        }
        if (!ok) {
          atomicOr(&elems[u.e].state[ST_ERROR], ERR_TIMEOUT);
          atomicOr(&abort_flag, 1);
          break;
        }
        mma_commit(&bar_dfull[b]);
        ++win;
      }
      // the MMAs must finish before tensor memory is released
      if (issued) mbar_wait(&bar_empty[last_stage % UNST], (last_stage / UNST) & 1, cleanup_polls);
    }
  } else if (warp < 2 + NSPLIT) {
    // ------------------------------------------------ transpose and split
    const int r = tid - 64;  // 0..127: grid row of the tile
    uint32_t stage = 0;
    int a = a0, ycur = -1;
    UElem u{};
      if (i0 < i1) u = uelem(elems, act, a, job);  // i0 < i1: a < nact
    for (int i = i0; i < i1 && !abort_flag; ++i) {
      while (tile0[a + 1] <= i) u = uelem(elems, act, ++a, job);
      bool ok = true;
      if (a != ycur) {
        // the B operand of the new element, once every MMA reading the
        // previous one has completed
        if (stage > 0) ok = mbar_wait(&bar_empty[(stage - 1) % UNST], ((stage - 1) / UNST) & 1, polls);
        if (ok) {
          const ElemDev<float>& E = elems[u.e];
          const int nq = u.nch * (UKC / 4);
          for (int t = r; t < u.N * nq; t += 32 * NSPLIT) {
            const int c = t / nq, q = t - c * nq;
            const int j = q >> 3, kq = q & 7;
            const int k0 = UKC * j + 4 * kq;
            const float4 x = make_float4(ycoef(E, u, job, k0, c), ycoef(E, u, job, k0 + 1, c),
                                         ycoef(E, u, job, k0 + 2, c), ycoef(E, u, job, k0 + 3, c));
            const float4 h = tf32_hi4(x);
            const uint32_t off = (uint32_t)(j * OPB_CHUNK) + sw_off(c, 4 * kq);
            *reinterpret_cast<float4*>(ybh + off) = h;
            *reinterpret_cast<float4*>(ybl + off) = tf32_lo4(x, h);
          }
          ycur = a;
        }
      }
      for (int j = 0; j < u.nch && ok; ++j, ++stage) {
        const int s = stage % UNST;
        ok = mbar_wait(&bar_full[s], (stage / UNST) & 1, polls);
        if (!ok || abort_flag) {
          ok = false;
          break;
        }
        unsigned char* stg = stages + (size_t)s * STAGE_BYTES_U;
        const float* src = reinterpret_cast<const float*>(stg);
        unsigned char* dh = stg + STG_BYTES;
        unsigned char* dl = dh + OPA_BYTES;
#pragma unroll
        for (int kq = 0; kq < UKC / 4; ++kq) {
          const int k0 = UKC * j + 4 * kq;
          float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
          if (k0 < u.K)  // whole quads: K is a multiple of 16
            x = make_float4(src[(4 * kq) * UM + r], src[(4 * kq + 1) * UM + r], src[(4 * kq + 2) * UM + r],
                            src[(4 * kq + 3) * UM + r]);
          const float4 h = tf32_hi4(x);
          const uint32_t off = sw_off(r, 4 * kq);
          *reinterpret_cast<float4*>(dh + off) = h;
          *reinterpret_cast<float4*>(dl + off) = tf32_lo4(x, h);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_conv[s]);
      }
      if (!ok) {
        atomicOr(&elems[u.e].state[ST_ERROR], ERR_TIMEOUT);
        atomicOr(&abort_flag, 1);
        break;
      }
    }
  } else {
    // ------------------------------------------------ epilogue
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    uint32_t win = 0;
    int a = a0;
    UElem u{};
      if (i0 < i1) u = uelem(elems, act, a, job);  // i0 < i1: a < nact
    for (int i = i0; i < i1; ++i) {
      while (tile0[a + 1] <= i) u = uelem(elems, act, ++a, job);
      const uint32_t b = win & 1;
      if (!mbar_wait(&bar_dfull[b], (win >> 1) & 1, polls)) {
        atomicOr(&elems[u.e].state[ST_ERROR], ERR_TIMEOUT);
        atomicOr(&abort_flag, 1);
        break;
      }
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const ElemDev<float>& E = elems[u.e];
      const int grow = (i - tile0[a]) * UM + row;
      const bool valid = grow < E.ng;
      const int sel_o = job.out_sel, sel_2 = job.out2_sel;
      float* O = E.blk[sel_o][sel_o < NDBL ? (u.par ^ job.out_next) : 0];
      float* O2 = job.from2 >= 0 ? E.blk[sel_2][sel_2 < NDBL ? (u.par ^ job.out2_next) : 0] : nullptr;
#pragma unroll
      for (int q = 0; q < UNMAX / 16; ++q) {
        if (16 * q >= u.N) break;
        float d0[16], d1[16];
        if (u.has0) {
          tmem_ld16(tmem + lane_base + b * UACC + (uint32_t)(16 * q), d0);
        } else {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) d0[jj] = 0.f;
        }
        if (u.has1) {
          tmem_ld16(tmem + lane_base + b * UACC + 64u + (uint32_t)(16 * q), d1);
        } else {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) d1[jj] = 0.f;
        }
        if (valid) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int c = 16 * q + jj;
            if (c >= u.m) break;
            float* o = O + (size_t)c * E.ng + grow;
            const float v = job.alpha * (d0[jj] + d1[jj]);
            *o = (job.beta == 0.f) ? v : v + job.beta * *o;
            if (O2) O2[(size_t)c * E.ng + grow] = d1[jj];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_dempty[b]);
      ++win;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_uencode = nullptr;
std::once_flag g_uencode_once;
int g_usms = 0;

}  // namespace

bool tf32_update_eligible(const BatchShape& s) {
  return s.max_m <= UNMAX && s.max_m > 0 && s.ng_mult4 && s.nel <= MAX_UPD_EL && s.nel > 0;
}

std::string encode_tf32_update_maps(const ElemDev<float>* h, int nel, void* host_out) {
  std::call_once(g_uencode_once, []() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_uencode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_uencode) return "cuTensorMapEncodeTiled is not available";
  unsigned char* out = static_cast<unsigned char*>(host_out);
  for (int e = 0; e < nel; ++e) {
    for (int idx = 0; idx < 10; ++idx) {
      const int sel = idx < 2 * NDBL ? idx / 2 : NDBL + (idx - 2 * NDBL);
      const int buf = idx < 2 * NDBL ? (idx & 1) : 0;
      void* ptr = h[e].blk[sel][buf];
      if (((uintptr_t)ptr & 15) || (h[e].ng & 3)) return "block not 16-byte aligned";
      cuuint64_t dims[2] = {(cuuint64_t)h[e].ng, (cuuint64_t)h[e].m};
      cuuint64_t strides[1] = {(cuuint64_t)h[e].ng * 4};
      cuuint32_t box[2] = {(cuuint32_t)UM, (cuuint32_t)UBOX};
      cuuint32_t estr[2] = {1, 1};
      CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out + ((size_t)e * 10 + idx) * 128);
      const CUresult r = g_uencode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    }
  }
  return "";
}

void init_tf32_update_kernel() {
  cudaFuncSetAttribute((const void*)tf32_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)UDYN_SMEM);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_usms, cudaDevAttrMultiProcessorCount, dev);
}

bool launch_tf32_update(const Batch<float>& b, const TsmmJob<float>& t, const void* d_maps, uint32_t polls,
                        cudaStream_t st) {
  if (!d_maps || !tf32_update_eligible(b.s)) return false;
  if (t.nin < 1 || t.nin > 3 || t.rows > 0 || t.ncols > 0 || t.ld_in > 0 || t.ycol != 0) return false;
  if (t.out.ptr || (t.from2 >= 0 && t.out2.ptr)) return false;
  if (t.y_id == Y_PTR && !t.y_ptr) return false;
  UpdJob j{};
  j.nin = t.nin;
  for (int i = 0; i < t.nin; ++i) {
    if (t.in[i].ptr) return false;
    j.sel[i] = t.in[i].sel;
    j.next[i] = t.in[i].next;
    j.needs_p[i] = t.needs_p[i];
    j.yrow[i] = t.yrow[i];
  }
  j.y_id = t.y_id;
  j.y_ptr = t.y_ptr;
  j.ldy = t.ldy;
  j.out_sel = t.out.sel;
  j.out_next = t.out.next;
  j.from2 = t.from2;
  j.out2_sel = t.from2 >= 0 ? t.out2.sel : 0;
  j.out2_next = t.from2 >= 0 ? t.out2.next : 0;
  j.alpha = (float)t.alpha;
  j.beta = (float)t.beta;
  const int G = g_usms > 0 ? g_usms : 148;
  tf32_update_kernel<<<G, UTHREADS, UDYN_SMEM, st>>>(b.d_elems, b.s.nel, static_cast<const unsigned char*>(d_maps),
                                                    j, polls ? polls : UDEFAULT_POLLS);
  return true;
}

}  // namespace dgdft
