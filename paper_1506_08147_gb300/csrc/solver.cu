// Host runtime of the ALB generator: context, memory admission, per-element
// device setup, the batched LOBPCG driver (one captured CUDA graph per
// iteration, replayed for all elements of a wave) and the C-ABI.
//
// Flow of dgdft_alb_solve (Sec. II.A; Sec. II.B "Generation of the ALB
// functions"): elements are admitted in waves that fit the device-memory
// budget; a wave runs LOBPCG for all its elements at once (inter-element
// parallelism of the paper becomes the grid's z dimension), then restricts
// the lowest J Ritz vectors to E_K and orthonormalises them in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dgdft_alb.h"
#include "../../include/dgdft_alb_steps.h"
#include "internal.h"
#include "learned.h"

using namespace dgdft;

namespace dgdft {
std::string cuda_err_string(cudaError_t e) { return std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e); }
template <class real>
void launch_proj_coef(const Batch<real>& b, BRef<real> src, int ncols, cudaStream_t st);
}  // namespace dgdft

namespace {

constexpr size_t ALIGN = 256;

struct ElemHost {
  dgdft_element_desc d{};
  // inputs, resident on the device once set
  double* d_veff = nullptr;  // N_g
  bool has_v = false;
  std::vector<int64_t> prow{0};
  std::vector<int32_t> pidx;
  std::vector<double> pval, pgamma;
  int proj_version = 0;
  double* d_x0 = nullptr;    // N_g x m
  bool has_x0 = false;
  bool x0_fresh = false;     // set_initial since the last solve / SCF step
  // results, on the device after a solve
  double* d_phi = nullptr;   // n_E x J
  double* d_eig = nullptr;   // J
  double* d_res = nullptr;   // J
  bool solved = false;
  std::vector<double> eig, resid, block;
  dgdft_solve_report rep{};
  int ng() const { return d.nx * d.ny * d.nz; }
  int ne() const { return (d.e_hi[0] - d.e_lo[0]) * (d.e_hi[1] - d.e_lo[1]) * (d.e_hi[2] - d.e_lo[2]); }
  double dv() const { return d.Lx * d.Ly * d.Lz / ng(); }
  void release() {
    for (double** p : {&d_veff, &d_x0, &d_phi, &d_eig, &d_res})
      if (*p) {
        cudaFree(*p);
        *p = nullptr;
      }
  }
};

bool plan_length(int n, FftPlan& p) {
  p.n = n;
  p.nstage = 0;
  int r = n;
  const int radices[4] = {4, 2, 3, 5};
  for (int q = 0; q < 4; ++q) {
    while (r % radices[q] == 0) {
      if (p.nstage >= MAX_STAGES) return false;
      p.radix[p.nstage++] = radices[q];
      r /= radices[q];
    }
  }
  return r == 1 && n >= 2;
}

std::vector<double> twiddles(int n, int count) {
  std::vector<double> t(2 * (size_t)count);
  for (int i = 0; i < count; ++i) {
    const double a = -2.0 * M_PI * (double)i / (double)n;
    t[2 * i] = std::cos(a);
    t[2 * i + 1] = std::sin(a);
  }
  return t;
}

std::vector<double> kinetic_axis(int n, double L, bool half) {
  const int cnt = half ? n / 2 + 1 : n;
  std::vector<double> g(cnt);
  for (int i = 0; i < cnt; ++i) {
    const int f = (half || i <= n / 2) ? i : i - n;
    const double k = 2.0 * M_PI * (double)std::abs(f) / L;
    g[i] = 0.5 * k * k;
  }
  return g;
}

// Grid frequencies of the element with |G|^2/2 <= ecut (the whole grid,
// both halves of every axis).
long long cutoff_set_size(const dgdft_element_desc& d, double ecut) {
  std::vector<double> gx = kinetic_axis(d.nx, d.Lx, false);
  const std::vector<double> gy = kinetic_axis(d.ny, d.Ly, false), gz = kinetic_axis(d.nz, d.Lz, false);
  std::sort(gx.begin(), gx.end());
  long long cnt = 0;
  for (double z : gz)
    for (double y : gy) cnt += std::upper_bound(gx.begin(), gx.end(), ecut - y - z) - gx.begin();
  return cnt;
}

// Device arena: one allocation carved into aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  void* take(size_t bytes) {
    const size_t off = (used + ALIGN - 1) / ALIGN * ALIGN;
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

struct Sizer {
  size_t total = 0;
  void add(size_t bytes) { total = (total + ALIGN - 1) / ALIGN * ALIGN + bytes; }
};

template <class real> struct Wave;

}  // namespace

struct dgdft_alb_ctx {
  dgdft_alb_config cfg{};
  std::vector<ElemHost> el;
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool solved_any = false;
  // waves kept resident between solves when every element fits in one
  void* cache = nullptr;
  void (*cache_free)(void*) = nullptr;
  // scratch of the restriction and orthonormalisation, kept between calls
  // (grown when a call needs more)
  void* ortho_buf = nullptr;
  size_t ortho_cap = 0;
  std::vector<int> cache_proj_version;
  ConvNet* net = nullptr;  // learned preconditioner, created on first use
  int wait_polls = 0;      // bounded device waits: polls before giving up (0: default)
  // autotuner: launch shapes per batch-shape key, read from and written to
  // the JSON file named by the config (empty path: no tuning, defaults)
  std::string tune_path;
  std::map<std::string, int> tune;
  bool tune_loaded = false;
  void tune_load() {
    if (tune_loaded || tune_path.empty()) return;
    tune_loaded = true;
    std::ifstream f(tune_path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    // a flat object of "key": integer pairs
    size_t p = 0;
    while ((p = t.find('"', p)) != std::string::npos) {
      const size_t q = t.find('"', p + 1);
      if (q == std::string::npos) break;
      const std::string key = t.substr(p + 1, q - p - 1);
      size_t c = t.find_first_not_of(" \t\r\n", q + 1);
      if (c == std::string::npos || t[c] != ':') {
        p = q + 1;
        continue;
      }
      char* end = nullptr;
      const long v = std::strtol(t.c_str() + c + 1, &end, 10);
      if (end != t.c_str() + c + 1) tune[key] = (int)v;
      p = (size_t)(end - t.c_str());
    }
  }
  void tune_save() const {
    if (tune_path.empty()) return;
    std::ofstream f(tune_path, std::ios::trunc);
    if (!f) return;
    f << "{";
    bool first = true;
    for (const auto& kv : tune) {
      f << (first ? "\n" : ",\n") << "  \"" << kv.first << "\": " << kv.second;
      first = false;
    }
    f << "\n}\n";
  }
  void drop_cache() {
    if (cache && cache_free) cache_free(cache);
    cache = nullptr;
    cache_proj_version.clear();
  }
  dgdft_status fail(dgdft_status s, const std::string& msg) {
    err = msg;
    return s;
  }
};


// Every host<->device copy runs on the context stream and completes before
// returning, so it is ordered with the library's kernels whatever the
// stream's flags.
static cudaError_t ctx_copy(dgdft_alb_ctx* ctx, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(ctx->stream);
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return ctx->fail(DGDFT_ECUDA, std::string(#call) + " -> " + \
                                                               cuda_err_string(e_)); \
  } while (0)

namespace {

int nchunk_rows(int ng) { return std::max(1, std::min(256, (ng + 4095) / 4096)); }

// Device footprint of one element in a wave of working precision `real`.
template <class real>
size_t elem_bytes(const ElemHost& h) {
  const dgdft_element_desc& d = h.d;
  const size_t ng = (size_t)h.ng(), m = (size_t)d.n_compute;
  const size_t nxh = d.nx / 2 + 1, nspec = nxh * d.ny * d.nz;
  const size_t np = h.pgamma.size(), nnz = h.pidx.size();
  Sizer s;
  s.add(ng * sizeof(real));                               // V
  s.add((sizeof(cplx_t<real>) + sizeof(double2)) * (d.nx / 2 + d.nx + d.ny + d.nz + 4));
  s.add(sizeof(double) * (nxh + d.ny + d.nz));
  s.add(sizeof(float) * (nxh + d.ny + d.nz + 3 * m * m) + 4 * ALIGN);
  s.add(sizeof(int) * (np + 1) + sizeof(int) * nnz + sizeof(real) * nnz + sizeof(double) * np);
  s.add(sizeof(int) * (d.nz + 1) + sizeof(int) * (3 * nnz + 1) + sizeof(real) * nnz);
  s.add(sizeof(int) * 4 * nnz);   // padded per-point copy (at most 4 nnz per point,
  s.add(sizeof(real) * 4 * nnz);  // so at most nnz points)
  s.add(sizeof(real) * np * m);
  for (int i = 0; i < 10; ++i) s.add(sizeof(real) * ng * m);
  s.add(sizeof(double2) * nspec * m);
  s.add(sizeof(double) * (18 * m * m + m * m + 3 * m * m + 3 * m + 2));
  s.add(sizeof(double) * rr_work_doubles(3 * (int)m, (int)m));
  s.add(sizeof(int) * STATE_WORDS);
  // the residual partial sums and the Gram partial buffer depend on the
  // wave's largest element and are added by Wave::build
  return s.total + 64 * ALIGN;
}

void default_x0(std::vector<double>& x, int elem);

// The FP32 stage's Gram products run on the tensor cores (TF32 split, TMA)
// unless the SIMT kernels are selected, when every element has m <= 48 and
// N_g a multiple of 4 (16-byte column starts for the copies).
inline bool tf32_selected(const dgdft_alb_config& c, const BatchShape& s) {
  return (c.bulk_kernels == 0 || c.bulk_kernels == 2) && tf32_gram_eligible(s);
}

template <class real> struct Wave {
  dgdft_alb_ctx* ctx = nullptr;
  std::vector<int> ids;
  std::vector<ElemDev<real>> h;
  Arena arena;
  ElemDev<real>* d_elems = nullptr;
  RRTask* d_rr_init = nullptr;
  RRTask* d_rr_lob = nullptr;
  double* partial = nullptr;
  size_t partial_cap = 0;
  Batch<real> batch;
  int rnchunk = 1;
  std::vector<int> h_state;
  // learned preconditioner buffers (FP32 waves with a network, uniform grids)
  bool learned = false;
  int gnz = 0, gny = 0, gnx = 0;
  float *nn_in = nullptr, *nn_out = nullptr, *nn_tmp0 = nullptr, *nn_tmp1 = nullptr;
  // Two half-batches iterated on two streams, the second half a
  // half-iteration behind: the Rayleigh-Ritz kernel of one half (one CTA per
  // element, bound by the FP64 pipe of few SMs) then runs beside the
  // bandwidth-bound kernels of the other half instead of leaving most SMs idle.
  struct SubView {
    Batch<real> batch;
    RRTask *rr_init = nullptr, *rr_lob = nullptr;
    double* partial = nullptr;
    size_t partial_cap = 0;
    const unsigned char* maps = nullptr;
    const unsigned char* umaps = nullptr;
  };
  // TMA tensor maps of every element's blocks (FP32 waves on the tensor-core
  // Gram), 10 x 128 bytes per element; nullptr when the SIMT Gram runs
  unsigned char* d_maps = nullptr;
  const unsigned char* maps = nullptr;  // of the current view
  // the same blocks' tensor maps for the tensor-core block updates (boxes of
  // 128 rows x 16 columns)
  unsigned char* d_umaps = nullptr;
  const unsigned char* umaps = nullptr;
  SubView full, sub[2];
  bool split = false;
  bool hx64 = false;            // capture H X' with the FP64 forward transform
  long long graph_kernels = 0;  // kernel nodes launched through graphs by run()
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Instantiated iteration graphs kept across runs (solves and SCF steps):
  // every pointer their nodes hold belongs to the wave, so they stay valid
  // for its life.  Keyed by what changes the nodes: the residual kernel's
  // iteration cap, the precise-H X' variant, the FP64 forward transform and
  // the restart budget.
  struct GraphSet {
    int maxit = 0, precise = 0, fwd = 0, restart = 0;
    cudaGraphExec_t exec = nullptr, exec2 = nullptr, pexec = nullptr, pexec2 = nullptr;
    long long nodes1 = 0, nodes2 = 0;
  };
  std::vector<GraphSet> graphs;

  ~Wave() {
    for (GraphSet& g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.exec2) cudaGraphExecDestroy(g.exec2);
      if (g.pexec) cudaGraphExecDestroy(g.pexec);
      if (g.pexec2) cudaGraphExecDestroy(g.pexec2);
    }
    if (arena.base) cudaFree(arena.base);
    for (float* p : {nn_in, nn_out, nn_tmp0, nn_tmp1})
      if (p) cudaFree(p);
    if (st2) cudaStreamDestroy(st2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }

  void use(const SubView& v) {
    batch = v.batch;
    d_rr_init = v.rr_init;
    d_rr_lob = v.rr_lob;
    partial = v.partial;
    partial_cap = v.partial_cap;
    maps = v.maps;
    umaps = v.umaps;
  }

  // Half-batch views; split only FP32 waves of >= 2 elements without the
  // learned preconditioner (its scratch is shared by the wave).
  dgdft_status setup_split() {
    full.batch = batch;
    full.rr_init = d_rr_init;
    full.rr_lob = d_rr_lob;
    full.partial = partial;
    full.partial_cap = partial_cap;
    full.maps = d_maps;
    maps = d_maps;
    full.umaps = d_umaps;
    umaps = d_umaps;
    const int nel = batch.s.nel;
    if (!std::is_same<real, float>::value || learned || nel < 2) return DGDFT_OK;
    const int h0 = nel / 2;
    const size_t per = partial_cap / nel;
    for (int k = 0; k < 2; ++k) {
      const int off = k ? h0 : 0, cnt = k ? nel - h0 : h0;
      SubView& v = sub[k];
      v.batch = batch;
      v.batch.d_elems = d_elems + off;
      v.batch.s.nel = cnt;
      v.rr_init = d_rr_init + off;
      v.rr_lob = d_rr_lob + off;
      v.partial = partial + per * off;
      v.partial_cap = per * cnt;
      v.maps = d_maps ? d_maps + (size_t)off * 10 * 128 : nullptr;
      v.umaps = d_umaps ? d_umaps + (size_t)off * 10 * 128 : nullptr;
    }
    CK(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    split = true;
    return DGDFT_OK;
  }

  dgdft_status setup_learned() {
    if (!std::is_same<real, float>::value || ctx->cfg.precond != DGDFT_PRECOND_LEARNED) return DGDFT_OK;
    if (!ctx->net || !ctx->net->ready) return ctx->fail(DGDFT_ESTATE, "learned preconditioner selected but no network");
    const dgdft_element_desc& d0 = ctx->el[ids[0]].d;
    for (int id : ids) {
      const dgdft_element_desc& d = ctx->el[id].d;
      if (d.nx != d0.nx || d.ny != d0.ny || d.nz != d0.nz) return DGDFT_OK;  // uneven grids: Teter only
    }
    gnz = d0.nz;
    gny = d0.ny;
    gnx = d0.nx;
    const size_t samples = (size_t)batch.s.nel * batch.s.max_m, ng = (size_t)gnx * gny * gnz;
    if (cudaMalloc(&nn_in, sizeof(float) * samples * 2 * ng) || cudaMalloc(&nn_out, sizeof(float) * samples * ng) ||
        cudaMalloc(&nn_tmp0, sizeof(float) * samples * 16 * ng) ||
        cudaMalloc(&nn_tmp1, sizeof(float) * samples * 16 * ng))
      return ctx->fail(DGDFT_ENOMEM, "learned preconditioner buffers");
    learned = true;
    return DGDFT_OK;
  }

  int restart_max = 0;  // see RRTask::restart_max (FP32 waves)

  dgdft_status build(dgdft_alb_ctx* c, const std::vector<int>& elem_ids, double cond_max, int restarts = 0) {
    restart_max = restarts;
    ctx = c;
    ids = elem_ids;
    const int nel = (int)ids.size();
    BatchShape s;
    s.nel = nel;
    for (int id : ids) {
      const ElemHost& eh = ctx->el[id];
      s.max_nz = std::max(s.max_nz, eh.d.nz);
      s.max_ny = std::max(s.max_ny, eh.d.ny);
      s.max_nxh = std::max(s.max_nxh, eh.d.nx / 2 + 1);
      s.max_nplane = std::max(s.max_nplane, (eh.d.nx / 2 + 1) * eh.d.ny);
      s.max_m = std::max(s.max_m, eh.d.n_compute);
      s.max_ng = std::max(s.max_ng, eh.ng());
      s.max_nproj = std::max(s.max_nproj, (int)eh.pgamma.size());
      s.ng_mult4 = s.ng_mult4 && (eh.ng() % 4 == 0);
    }
    {
      const dgdft_element_desc& d0 = ctx->el[ids[0]].d;
      bool uni = true;
      for (int id : ids) {
        const dgdft_element_desc& d = ctx->el[id].d;
        uni = uni && d.nx == d0.nx && d.ny == d0.ny && d.nz == d0.nz;
      }
      if (uni) {
        s.uni_nx = d0.nx;
        s.uni_ny = d0.ny;
        s.uni_nz = d0.nz;
      }
    }
    // the refinement (FP64) stage of the mixed form takes its Gram products
    // in double-float arithmetic; the plain FP64 solver stays on the FP64 pipe
    s.dfloat = std::is_same<real, double>::value && ctx->cfg.precision == DGDFT_PREC_MIXED;
    rnchunk = nchunk_rows(s.max_ng);
    const size_t tiles = ((s.max_m + 63) / 64) * ((s.max_m + 63) / 64);
    const size_t pcap = (size_t)nel * ((s.max_ng + 2047) / 2048) * 12 * tiles * 4096;
    size_t total = 0;
    for (int id : ids) {
      total += elem_bytes<real>(ctx->el[id]);
      total += sizeof(double) * (size_t)ctx->el[id].d.n_compute * rnchunk * 4 + ALIGN;  // rpart
    }
    total += sizeof(double) * pcap + ALIGN;
    total += (sizeof(ElemDev<real>) + 2 * sizeof(RRTask)) * nel + 4 * ALIGN;
    const bool want_maps = std::is_same<real, float>::value && tf32_selected(ctx->cfg, s);
    if (want_maps) total += 2 * ((size_t)nel * 10 * 128 + ALIGN);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, total);
    if (e != cudaSuccess) return ctx->fail(DGDFT_ENOMEM, "device allocation of a wave failed: " + cuda_err_string(e));
    arena.base = (char*)p;
    arena.cap = total;
    // Gram partials: shared by the wave
    partial_cap = pcap;
    partial = (double*)arena.take(partial_cap * sizeof(double));
    d_elems = (ElemDev<real>*)arena.take(sizeof(ElemDev<real>) * nel);
    d_rr_init = (RRTask*)arena.take(sizeof(RRTask) * nel);
    d_rr_lob = (RRTask*)arena.take(sizeof(RRTask) * nel);
    h.resize(nel);
    std::vector<RRTask> rr_init(nel), rr_lob(nel);
    h_state.assign((size_t)nel * STATE_WORDS, 0);
    for (int i = 0; i < nel; ++i) {
      dgdft_status st = setup_elem(i, ctx->el[ids[i]]);
      if (st != DGDFT_OK) return st;
      ElemDev<real>& E = h[i];
      RRTask t{};
      t.A = E.gram;
      t.B = E.gram + (size_t)9 * E.m * E.m;
      t.ld = 3 * E.m;
      t.mode = RR_INITIAL;
      t.n_fixed = E.m;
      t.m = E.m;
      t.Y = E.Y;
      t.Yf = E.Yf;
      t.ldy = 3 * E.m;
      t.theta = E.theta;
      t.work = E.rr_work;
      t.state = E.state;
      t.cond_max = cond_max;
      t.restart_max = 0;
      rr_init[i] = t;
      t.restart_max = restarts;
      t.mode = RR_LOBPCG;
      rr_lob[i] = t;
    }
    if (want_maps) {
      // tensor maps need the blocks' device addresses: encoded here, once
      std::vector<unsigned char> hm((size_t)nel * 10 * 128);
      std::string err;
      if constexpr (std::is_same<real, float>::value) err = encode_tf32_gram_maps(h.data(), nel, hm.data());
      unsigned char* dm = (unsigned char*)arena.take(hm.size());
      if (err.empty() && dm) {
        CK(ctx_copy(ctx, dm, hm.data(), hm.size(), cudaMemcpyHostToDevice));
        d_maps = dm;
      }
      err.clear();
      if constexpr (std::is_same<real, float>::value)
        if (ctx->cfg.bulk_kernels == 2 && tf32_update_eligible(s))
          err = encode_tf32_update_maps(h.data(), nel, hm.data());
        else
          err = "not selected";
      unsigned char* du = (unsigned char*)arena.take(hm.size());
      if (err.empty() && du) {
        CK(ctx_copy(ctx, du, hm.data(), hm.size(), cudaMemcpyHostToDevice));
        d_umaps = du;
      }
    }
    CK(ctx_copy(ctx, d_elems, h.data(), sizeof(ElemDev<real>) * nel, cudaMemcpyHostToDevice));
    CK(ctx_copy(ctx, d_rr_init, rr_init.data(), sizeof(RRTask) * nel, cudaMemcpyHostToDevice));
    CK(ctx_copy(ctx, d_rr_lob, rr_lob.data(), sizeof(RRTask) * nel, cudaMemcpyHostToDevice));
    batch.d_elems = d_elems;
    batch.s = s;
    if constexpr (std::is_same<real, float>::value) {
      dgdft_status ts = autotune_update();
      if (ts != DGDFT_OK) return ts;
    }
    dgdft_status ls = setup_learned();
    if (ls != DGDFT_OK) return ls;
    return setup_split();
  }

  // Autotuner: the FP32 block update's 128-row tiles per CTA for this batch
  // shape, from the context's cache or, when missing, timed here on the
  // wave's own blocks (every element marked active with P for the timing,
  // the state words restored after; the output is the next X buffer, scratch
  // before the first iteration).  The choice changes no result.
  dgdft_status autotune_update() {
    if (ctx->tune_path.empty()) return DGDFT_OK;
    ctx->tune_load();
    const BatchShape& s = batch.s;
    const std::string key = "tsmm_rows_tiles nel=" + std::to_string(s.nel) + " m=" + std::to_string(s.max_m) +
                            " ng=" + std::to_string(s.max_ng);
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end() && it->second > 0) {
      batch.s.tsmm_tiles = it->second;
      return DGDFT_OK;
    }
    const int nel = s.nel;
    std::vector<int> saved((size_t)nel * STATE_WORDS), on((size_t)nel * STATE_WORDS, 0);
    for (int i = 0; i < nel; ++i)
      CK(ctx_copy(ctx, &saved[(size_t)i * STATE_WORDS], h[i].state, sizeof(int) * STATE_WORDS,
                  cudaMemcpyDeviceToHost));
    for (int i = 0; i < nel; ++i) {
      on[(size_t)i * STATE_WORDS + ST_ACTIVE] = 1;
      on[(size_t)i * STATE_WORDS + ST_HAS_P] = 1;
      CK(ctx_copy(ctx, h[i].state, &on[(size_t)i * STATE_WORDS], sizeof(int) * STATE_WORDS,
                  cudaMemcpyHostToDevice));
    }
    TsmmJob<real> t;
    t.nin = 3;
    t.in[0] = bref<real>(BX);
    t.in[1] = bref<real>(BW);
    t.in[2] = bref<real>(BP);
    t.yrow[1] = 1;
    t.yrow[2] = 2;
    t.needs_p[2] = 1;
    t.out = bref<real>(BX, 1);
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = 8;
    float best_ms = 1e30f;
    for (int tiles : {2, 4, 8, 16}) {
      batch.s.tsmm_tiles = tiles;
      launch_tsmm<real>(batch, t, st);
      CK(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) launch_tsmm<real>(batch, t, st);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = tiles;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    for (int i = 0; i < nel; ++i)
      CK(ctx_copy(ctx, h[i].state, &saved[(size_t)i * STATE_WORDS], sizeof(int) * STATE_WORDS,
                  cudaMemcpyHostToDevice));
    batch.s.tsmm_tiles = best;
    ctx->tune[key] = best;
    ctx->tune_save();
    return DGDFT_OK;
  }

  template <class T> T* take(size_t count) { return (T*)arena.take(sizeof(T) * std::max<size_t>(count, 1)); }

  template <class T> dgdft_status put(T* dst, const T* src, size_t count) {
    if (count) CK(ctx_copy(ctx, dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    return DGDFT_OK;
  }

  dgdft_status setup_elem(int i, const ElemHost& eh) {
    using C = cplx_t<real>;
    const dgdft_element_desc& d = eh.d;
    ElemDev<real>& E = h[i];
    std::memset(&E, 0, sizeof(E));
    E.nx = d.nx;
    E.ny = d.ny;
    E.nz = d.nz;
    E.ng = eh.ng();
    E.nh = d.nx / 2;
    E.nxh = d.nx / 2 + 1;
    E.nspec = E.nxh * d.ny * d.nz;
    E.m = d.n_compute;
    E.J = d.n_keep;
    E.scale = 2.0 / (double)E.ng;
    E.tol = ctx->cfg.tol;
    E.ecut = ctx->cfg.ecut;
    plan_length(E.nh, E.px);
    plan_length(d.ny, E.py);
    plan_length(d.nz, E.pz);
    const size_t ng = E.ng, m = E.m;
    // potential: converted from the resident FP64 copy at every solve
    E.V = take<real>(ng);
    // twiddles, working precision and FP64
    auto put_tw = [&](int n, int count, int axis) -> bool {
      std::vector<double> t = twiddles(n, count);
      std::vector<C> tc(count);
      for (int q = 0; q < count; ++q) tc[q] = cmake<C>((real)t[2 * q], (real)t[2 * q + 1]);
      C* dp = take<C>(count);
      if (!dp || put(dp, tc.data(), count) != DGDFT_OK) return false;
      E.tw[axis] = dp;
      if (sizeof(real) == sizeof(double)) {
        E.tw64[axis] = reinterpret_cast<const double2*>(dp);
        // FP32-pair copy for double-float FFT passes (fits the FP64 table
        // budget that FP64 waves do not use)
        std::vector<float4> tf(count);
        for (int q = 0; q < count; ++q) {
          const double re = t[2 * q], im = t[2 * q + 1];
          const float rh = (float)re, ih = (float)im;
          tf[q] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
        }
        float4* fp = take<float4>(count);
        if (!fp || put(fp, tf.data(), count) != DGDFT_OK) return false;
        E.twdf[axis] = fp;
      } else {
        std::vector<double2> td(count);
        for (int q = 0; q < count; ++q) td[q] = make_double2(t[2 * q], t[2 * q + 1]);
        double2* dd = take<double2>(count);
        if (!dd || put(dd, td.data(), count) != DGDFT_OK) return false;
        E.tw64[axis] = dd;
      }
      return true;
    };
    if (!put_tw(E.nh, E.nh, TW_H) || !put_tw(d.nx, E.nh + 1, TW_X) || !put_tw(d.ny, d.ny, TW_Y) ||
        !put_tw(d.nz, d.nz, TW_Z))
      return ctx->fail(DGDFT_ECUDA, "twiddle upload");
    auto put_g = [&](const std::vector<double>& g) -> const double* {
      double* dp = take<double>(g.size());
      if (put(dp, g.data(), g.size()) != DGDFT_OK) return nullptr;
      return dp;
    };
    E.gx2 = put_g(kinetic_axis(d.nx, d.Lx, true));
    E.gy2 = put_g(kinetic_axis(d.ny, d.Ly, false));
    E.gz2 = put_g(kinetic_axis(d.nz, d.Lz, false));
    if (!E.gx2 || !E.gy2 || !E.gz2) return DGDFT_ECUDA;
    auto put_gf = [&](const std::vector<double>& g) -> const float* {
      std::vector<float> gf(g.begin(), g.end());
      float* dp = take<float>(gf.size());
      if (put(dp, gf.data(), gf.size()) != DGDFT_OK) return nullptr;
      return dp;
    };
    E.gx2f = put_gf(kinetic_axis(d.nx, d.Lx, true));
    E.gy2f = put_gf(kinetic_axis(d.ny, d.Ly, false));
    E.gz2f = put_gf(kinetic_axis(d.nz, d.Lz, false));
    if (!E.gx2f || !E.gy2f || !E.gz2f) return DGDFT_ECUDA;
    // projectors, CSR by projector
    const int np = (int)eh.pgamma.size();
    const size_t nnz = eh.pidx.size();
    E.n_proj = np;
    {
      std::vector<int> pp(np + 1);
      for (int q = 0; q <= np; ++q) pp[q] = (int)eh.prow[q];
      std::vector<real> pv(eh.pval.begin(), eh.pval.end());
      int* dpp = take<int>(np + 1);
      int* dpi = take<int>(nnz);
      real* dpv = take<real>(nnz);
      double* dpg = take<double>(np);
      if (put(dpp, pp.data(), np + 1) || put(dpi, eh.pidx.data(), nnz) || put(dpv, pv.data(), nnz) ||
          put(dpg, eh.pgamma.data(), (size_t)np))
        return DGDFT_ECUDA;
      E.p_ptr = dpp;
      E.p_idx = dpi;
      E.p_val = dpv;
      E.p_gamma = dpg;
      // grouped by grid point: (idx, proj, gamma * val), sorted by idx
      std::vector<std::pair<int, int>> ent(nnz);  // (idx, position)
      std::vector<int> owner(nnz);
      for (int q = 0; q < np; ++q)
        for (int64_t k = eh.prow[q]; k < eh.prow[q + 1]; ++k) owner[k] = q;
      for (size_t k = 0; k < nnz; ++k) ent[k] = {eh.pidx[k], (int)k};
      std::sort(ent.begin(), ent.end());
      std::vector<int> s_off, s_ptr{0}, s_proj(nnz), s_plane(d.nz + 1, 0);
      std::vector<real> s_gv(nnz);
      const int plane = d.nx * d.ny;
      for (size_t k = 0; k < nnz; ++k) {
        const int g = ent[k].first, pos = ent[k].second;
        if (k == 0 || g != ent[k - 1].first) {
          if (k) s_ptr.push_back((int)k);
          s_off.push_back(g % plane);
          s_plane[g / plane + 1] += 1;
        }
        s_proj[k] = owner[pos];
        s_gv[k] = (real)(eh.pgamma[owner[pos]] * eh.pval[pos]);
      }
      if (nnz) s_ptr.push_back((int)nnz);
      for (int z = 0; z < d.nz; ++z) s_plane[z + 1] += s_plane[z];
      E.n_sup = (int)s_off.size();
      int* dsp = take<int>(d.nz + 1);
      int* dso = take<int>(s_off.size());
      int* dsptr = take<int>(s_ptr.size());
      int* dspj = take<int>(nnz);
      real* dsg = take<real>(nnz);
      if (put(dsp, s_plane.data(), s_plane.size()) || put(dso, s_off.data(), s_off.size()) ||
          put(dsptr, s_ptr.data(), s_ptr.size()) || put(dspj, s_proj.data(), nnz) || put(dsg, s_gv.data(), nnz))
        return DGDFT_ECUDA;
      E.s_plane = dsp;
      E.s_off = dso;
      E.s_ptr = dsptr;
      E.s_proj = dspj;
      E.s_gv = dsg;
      // fixed-width copy (4 per point) when every point has at most 4
      int kmax = 0;
      for (size_t p = 0; p + 1 < s_ptr.size(); ++p) kmax = std::max(kmax, s_ptr[p + 1] - s_ptr[p]);
      E.s_proj4 = nullptr;
      E.s_gv4 = nullptr;
      if (kmax <= 4 && !s_off.empty()) {
        std::vector<int> pj4(4 * s_off.size(), 0);
        std::vector<real> gv4(4 * s_off.size(), (real)0);
        for (size_t p = 0; p + 1 < s_ptr.size(); ++p)
          for (int q = s_ptr[p]; q < s_ptr[p + 1]; ++q) {
            pj4[4 * p + (q - s_ptr[p])] = s_proj[q];
            gv4[4 * p + (q - s_ptr[p])] = s_gv[q];
          }
        int* d4p = take<int>(pj4.size());
        real* d4g = take<real>(gv4.size());
        if (put(d4p, pj4.data(), pj4.size()) || put(d4g, gv4.data(), gv4.size())) return DGDFT_ECUDA;
        E.s_proj4 = d4p;
        E.s_gv4 = d4g;
      }
      E.Ccoef = take<real>((size_t)np * m);
    }
    for (int b = 0; b < NBLK; ++b) {
      E.blk[b][0] = take<real>(ng * m);
      E.blk[b][1] = (b < NDBL) ? take<real>(ng * m) : E.blk[b][0];
    }
    E.Z = take<double2>((size_t)E.nspec * m);  // FP64 intermediate of the forward transform
    E.gram = take<double>(18 * m * m);
    E.gxw = take<double>(m * m);
    E.Y = take<double>(3 * m * m);
    E.Yf = std::is_same<real, float>::value ? take<float>(3 * m * m) : nullptr;
    E.theta = take<double>(m);
    E.res = take<double>(m);
    E.tkin = take<double>(m);
    E.sigma = take<double>(2);
    E.rr_work = take<double>(rr_work_doubles(3 * (int)m, (int)m));
    E.rpart = take<double>(m * rnchunk * 4);
    E.state = take<int>(STATE_WORDS);
    if (!E.state || !E.rpart || !E.rr_work || !E.Z || !E.sigma)
      return ctx->fail(DGDFT_ENOMEM, "wave arena exhausted");
    {
      const double zero2[2] = {0.0, 0.0};
      if (put(E.sigma, zero2, 2) != DGDFT_OK) return DGDFT_ECUDA;
    }
    return DGDFT_OK;
  }

  dgdft_status load_potential() {
    for (size_t i = 0; i < ids.size(); ++i)
      launch_convert<double, real>(ctx->el[ids[i]].d_veff, const_cast<real*>(h[i].V), (size_t)h[i].ng,
                                   ctx->stream);
    CK(cudaGetLastError());
    return DGDFT_OK;
  }

  // Working-precision copies of V_eff and X0 from the resident FP64 inputs;
  // warm (SCF steps): an FP64 device block per element to start from instead.
  dgdft_status load_inputs(const std::vector<const double*>* warm = nullptr) {
    dgdft_status ps = load_potential();
    if (ps != DGDFT_OK) return ps;
    for (size_t i = 0; i < ids.size(); ++i) {
      ElemHost& eh = ctx->el[ids[i]];
      ElemDev<real>& E = h[i];
      const size_t n = (size_t)E.ng * E.m;
      if (warm) {
        const double* src = (*warm)[i];
        if ((const void*)src != (const void*)E.blk[BX][0]) launch_convert<double, real>(src, E.blk[BX][0], n, ctx->stream);
      } else if (eh.has_x0) {
        launch_convert<double, real>(eh.d_x0, E.blk[BX][0], n, ctx->stream);
      } else {
        std::vector<double> x0(n);
        default_x0(x0, ids[i]);
        double* tmp = nullptr;
        CK(cudaMalloc(&tmp, n * sizeof(double)));
        cudaError_t e = ctx_copy(ctx, tmp, x0.data(), n * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
          launch_convert<double, real>(tmp, E.blk[BX][0], n, ctx->stream);
          e = cudaStreamSynchronize(ctx->stream);
        }
        cudaFree(tmp);
        if (e != cudaSuccess) return ctx->fail(DGDFT_ECUDA, "initial block: " + cuda_err_string(e));
      }
    }
    CK(cudaGetLastError());
    return DGDFT_OK;
  }

  // resume: elements already converged stay inactive with their results
  dgdft_status reset_states(double tol, bool resume = false) {
    const int nel = (int)ids.size();
    for (int i = 0; i < nel; ++i) {
      int* s = &h_state[(size_t)i * STATE_WORDS];
      const bool keep = resume && s[ST_CONVERGED];
      if (!keep) {
        std::fill(s, s + STATE_WORDS, 0);
        s[ST_ACTIVE] = 1;
        s[ST_TETER] = learned ? 0 : 1;
        CK(cudaMemsetAsync(h[i].sigma, 0, 2 * sizeof(double), ctx->stream));
      }
      h[i].tol = tol;
    }
    CK(ctx_copy(ctx, d_elems, h.data(), sizeof(ElemDev<real>) * nel, cudaMemcpyHostToDevice));
    for (int i = 0; i < nel; ++i)
      CK(ctx_copy(ctx, h[i].state, &h_state[(size_t)i * STATE_WORDS], sizeof(int) * STATE_WORDS,
                    cudaMemcpyHostToDevice));
    return DGDFT_OK;
  }

  dgdft_status read_states() {
    for (size_t i = 0; i < ids.size(); ++i)
      CK(cudaMemcpyAsync(&h_state[i * STATE_WORDS], h[i].state, sizeof(int) * STATE_WORDS,
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DGDFT_OK;
  }

  bool fwd64() const { return ctx->cfg.h_fp64_forward == 1; }

  // W = T(R): the learned network for elements that use it, Teter for the rest
  void precondition(cudaStream_t st) {
    if constexpr (std::is_same<real, float>::value) {
      if (learned) {
        learned_precondition(batch, *ctx->net, rnchunk, gnz, gny, gnx, nn_in, nn_out, nn_tmp0, nn_tmp1, st);
        launch_teter<real>(batch, bref<real>(BW), bref<real>(BW), nullptr, 0, st, 1);
        return;
      }
    }
    launch_teter<real>(batch, bref<real>(BW), bref<real>(BW), nullptr, 0, st);
  }
  const bool trace_ = std::getenv("DGDFT_TRACE") != nullptr;

  // Tensor-core Gram of the FP32 stage (mode 0: the 12 LOBPCG blocks, mode
  // 1: X^T W); returns false when the SIMT kernel must run.
  bool tc_gram(int mode, cudaStream_t st) {
    if constexpr (std::is_same<real, float>::value) {
      if (maps) return launch_tf32_gram(batch, maps, mode, partial, partial_cap, (uint32_t)ctx->wait_polls, st);
    }
    (void)mode;
    (void)st;
    return false;
  }

  // Block update out = alpha sum in_i Y_i + beta out: tensor cores in the
  // FP32 stage when selected (the TF32-split tcgen05 kernel), else SIMT.
  void update(const TsmmJob<real>& t, cudaStream_t st) {
    if constexpr (std::is_same<real, float>::value) {
      if (umaps && launch_tf32_update(batch, t, umaps, (uint32_t)ctx->wait_polls, st)) return;
    }
    launch_tsmm<real>(batch, t, st);
  }

  GramJob<real> gram12() const {
    GramJob<real> g;
    // A(i, j) for block(i) < block(j) is taken as (H s_i)^T s_j, H on the
    // earlier block: (H x)^T w = theta x^T w + r^T w is small, so its rounding
    // is small too, while x^T (H w) sums large terms that cancel.
    const int A_[6][4] = {{BHX, BX, 0, 0}, {BHX, BW, 0, 1}, {BHX, BP, 0, 2},
                          {BHW, BW, 1, 1}, {BHW, BP, 1, 2}, {BHP, BP, 2, 2}};
    const int B_[6][4] = {{BX, BX, 0, 0}, {BX, BW, 0, 1}, {BX, BP, 0, 2},
                          {BW, BW, 1, 1}, {BW, BP, 1, 2}, {BP, BP, 2, 2}};
    g.npairs = 12;
    for (int q = 0; q < 6; ++q) {
      for (int h2 = 0; h2 < 2; ++h2) {
        const int(*T)[4] = h2 ? B_ : A_;
        const int k = q + 6 * h2;
        g.a[k] = bref<real>(T[q][0]);
        g.b[k] = bref<real>(T[q][1]);
        g.needs_p[k] = (T[q][0] == BP || T[q][0] == BHP || T[q][1] == BP || T[q][1] == BHP);
        g.out_id[k] = h2 ? OUT_GRAM_B : OUT_GRAM_A;
        g.brow[k] = T[q][2];
        g.bcol[k] = T[q][3];
      }
    }
    return g;
  }

  // X^T W (into gxw) and the 12 pencil blocks (into gram): tensor cores in
  // the FP32 stage when selected, else the split-K SIMT kernels
  void gram_xtw(cudaStream_t st) {
    if (tc_gram(1, st)) return;
    GramJob<real> g;
    g.npairs = 1;
    g.a[0] = bref<real>(BX);
    g.b[0] = bref<real>(BW);
    g.needs_p[0] = 0;
    g.out_id[0] = OUT_GXW;
    g.brow[0] = g.bcol[0] = 0;
    launch_gram<real>(batch, g, partial, partial_cap, st);
  }
  void gram_pencil(cudaStream_t st) {
    if (!tc_gram(0, st)) launch_gram<real>(batch, gram12(), partial, partial_cap, st);
  }

  // Sphere-cutoff planewave set (a context with ecut > 0): the blocks stay
  // in the span of the set, so the Gram products of the unprojected H equal
  // those of the Galerkin problem.  The starting block is projected; W =
  // T(P R) keeps the set because the Teter multiplier is diagonal in G.
  // X' = [X W P] Y and P' = [W P] Y_wp are projected again before their H
  // applies: each FFT round trip leaves a rounding's worth of a column
  // outside the set (~1e-16 in FP64), which coefficients Y of an
  // ill-conditioned pencil would multiply (measured: 3e-10 after 45 FP64
  // iterations without it) and which would reach the Ritz values through the
  // Gram products.  In the FP32 stage HP' stays the update [HW HP] Y_wp, so
  // it differs from H of the projected P' by H of the removed part, the size
  // of that update's own FP32 rounding.
  bool cutoff() const { return ctx->cfg.ecut > 0.0; }
  void project_block(int sel, cudaStream_t st, int next = 0) {
    launch_project(batch, bref<real>(sel, next), bref<real>(sel, next), 0, st);
  }
  // R (in W) -> P R, and its norm |P R| in place of |R| in the residual sums
  void project_residual(cudaStream_t st) {
    launch_project(batch, bref<real>(BW), bref<real>(BW), 0, st);
    launch_rnorm(batch, rnchunk, st);
  }

  void enqueue_initial(cudaStream_t st) {
    if (cutoff()) project_block(BX, st);
    launch_apply_h<real>(batch, bref<real>(BX), bref<real>(BHX), 0, st, fwd64());
    GramJob<real> g;
    g.npairs = 2;
    g.a[0] = bref<real>(BX);
    g.b[0] = bref<real>(BHX);
    g.out_id[0] = OUT_GRAM_A;
    g.a[1] = bref<real>(BX);
    g.b[1] = bref<real>(BX);
    g.out_id[1] = OUT_GRAM_B;
    for (int k = 0; k < 2; ++k) g.needs_p[k] = g.brow[k] = g.bcol[k] = 0;
    launch_gram<real>(batch, g, partial, partial_cap, st);
    // double-float reduction in the FP32 stage and in the mixed form's
    // FP64-accurate stage (its pencils carry the double-float Gram's ~2^-44
    // rounding; the reduction's ~2^-46 adds nothing), FP64 otherwise
    launch_rr(d_rr_init, batch.s.nel, st, batch.s.max_m, batch.s.max_m,
              std::is_same<real, float>::value || batch.s.dfloat);
    TsmmJob<real> t;
    t.nin = 1;
    t.in[0] = bref<real>(BX);
    t.out = bref<real>(BX, 1);
    update(t, st);
    t.in[0] = bref<real>(BHX);
    t.out = bref<real>(BHX, 1);
    update(t, st);
    launch_iter_finish<real>(batch, 0, st);
  }

  void enqueue_iteration(cudaStream_t st, int maxit) {
    enqueue_front(st, maxit);
    enqueue_back(st);
  }

  // Residual, preconditioner, W and HW, Gram products (operations 1, 2, 5).
  void enqueue_front(cudaStream_t st, int maxit) {
    if (batch.s.max_nproj > 0) launch_proj_coef<real>(batch, bref<real>(BX), 0, st);
    launch_residual<real>(batch, rnchunk, st);
    if (cutoff()) project_residual(st);
    launch_post_residual<real>(batch, rnchunk, maxit, st);
    if (std::is_same<real, float>::value) launch_shift<real>(batch, st);
    precondition(st);
    {
      gram_xtw(st);
      TsmmJob<real> t;
      t.nin = 1;
      t.in[0] = bref<real>(BX);
      t.y_id = Y_GXW;
      t.out = bref<real>(BW);
      t.alpha = -1.0;
      t.beta = 1.0;
      update(t, st);
    }
    launch_apply_h<real>(batch, bref<real>(BW), bref<real>(BHW), 0, st, fwd64());
    gram_pencil(st);
  }

  // Rayleigh-Ritz and the block updates (operations 3, 4; H X for FP32).
  void enqueue_back(cudaStream_t st) {
    launch_rr(d_rr_lob, batch.s.nel, st, 3 * batch.s.max_m, batch.s.max_m,
              std::is_same<real, float>::value || batch.s.dfloat);
    {
      TsmmJob<real> t;
      t.nin = 3;
      t.in[0] = bref<real>(BX);
      t.in[1] = bref<real>(BW);
      t.in[2] = bref<real>(BP);
      t.yrow[0] = 0;
      t.yrow[1] = 1;
      t.yrow[2] = 2;
      t.needs_p[2] = 1;
      t.out = bref<real>(BX, 1);
      constexpr bool f32 = std::is_same<real, float>::value;
      if (f32) {
        // P' = [W P] Y_wp is the partial sum on the way to X' = X Y_x + P'
        t.from2 = 1;
        t.out2 = bref<real>(BP, 1);
      }
      update(t, st);
      t.from2 = -1;
      if (std::is_same<real, double>::value) {
        // FP64: H X' by the FFT (three FP64 passes cost less than the FP64
        // block update [HX HW HP] Y on the FP64 pipe)
        if (cutoff()) project_block(BX, st, 1);
        launch_apply_h<real>(batch, bref<real>(BX, 1), bref<real>(BHX, 1), 0, st, false);
      } else {
        // FP32: HX is recomputed as H X rather than updated as [HX HW HP] Y,
        // whose rounding grows with |Y| |HW| once [X W P] is nearly dependent
        // and would leave HX inconsistent with X (the residual then stalls or
        // diverges near 1e-4 Ha)
        if (restart_max > 0) launch_restart<real>(batch, st);
        if (cutoff()) {
          project_block(BX, st, 1);
          project_block(BP, st, 1);
        }
        launch_apply_h<real>(batch, bref<real>(BX, 1), bref<real>(BHX, 1), 0, st, fwd64() || hx64);
      }
      TsmmJob<real> u;
      u.nin = 2;
      u.in[0] = bref<real>(BW);
      u.in[1] = bref<real>(BP);
      u.yrow[0] = 1;
      u.yrow[1] = 2;
      u.needs_p[1] = 1;
      u.out = bref<real>(BP, 1);
      if (!f32) {
        launch_tsmm<real>(batch, u, st);
        // H P' by the FFT, as H X'
        if (cutoff()) project_block(BP, st, 1);
        launch_apply_h<real>(batch, bref<real>(BP, 1), bref<real>(BHP, 1), 0, st, false);
      } else {
        u.in[0] = bref<real>(BHW);
        u.in[1] = bref<real>(BHP);
        u.out = bref<real>(BHP, 1);
        update(u, st);
      }
    }
    launch_iter_finish<real>(batch, 1, st);
  }

  // LOBPCG for every element of the wave; stall_window > 0 stops an element
  // whose max residual has stopped improving over that many polls.
  // FP64 check of the current block without iterating: H X in the wave's
  // arithmetic, Rayleigh quotients as theta, residuals and convergence.
  dgdft_status verify(double tol) {
    cudaStream_t st = ctx->stream;
    dgdft_status s = reset_states(tol);
    if (s != DGDFT_OK) return s;
    // the FP32 stage's block, projected by the FP64 stage's mask
    if (cutoff()) project_block(BX, st);
    launch_apply_h<real>(batch, bref<real>(BX), bref<real>(BHX), 0, st, fwd64());
    launch_theta<real>(batch, rnchunk, 0, st);
    launch_residual<real>(batch, rnchunk, st);
    launch_theta<real>(batch, rnchunk, 1, st);
    if (batch.s.max_nproj > 0) launch_proj_coef<real>(batch, bref<real>(BX), 0, st);
    launch_residual<real>(batch, rnchunk, st);
    if (cutoff()) project_residual(st);
    launch_post_residual<real>(batch, rnchunk, 1 << 30, st);
    CK(cudaGetLastError());
    return read_states();
  }

  // precise_below > 0 (FP32 waves): once the median active element's residual
  // is below it, H X' is computed with the FP64 forward transform, whose
  // rounding no longer dominates the residual; the FP32 stage can then reach
  // tol.
  dgdft_status run(double tol, int maxit, int stall_window, std::vector<double>* res_out, int refresh_every = 0,
                   bool resume = false, double precise_below = 0.0, double stall_gain = 0.95) {
    cudaStream_t st = ctx->stream;
    const auto tr0 = std::chrono::steady_clock::now();
    auto trace_ms = [&]() { return 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - tr0).count(); };
    dgdft_status s = reset_states(tol, resume);
    if (s != DGDFT_OK) return s;
    if (trace_) std::fprintf(stderr, "[dgdft] run: states reset at %.2f ms\n", trace_ms());
    enqueue_initial(st);
    CK(cudaGetLastError());
    if (trace_) {
      cudaStreamSynchronize(st);
      std::fprintf(stderr, "[dgdft] run: initial Rayleigh-Ritz done at %.2f ms\n", trace_ms());
    }
    cudaGraphExec_t exec = nullptr, exec2 = nullptr;
    long long nodes1 = 0, nodes2 = 0;
    cudaError_t ce = cudaSuccess;
    // graphs of an earlier run with the same key are launched again (the
    // learned preconditioner's buffers belong to the context: not cached)
    const int want_precise = (precise_below > 0.0 && !fwd64()) ? 1 : 0;
    const bool cacheable = !learned;
    GraphSet* cached = nullptr;
    if (cacheable)
      for (GraphSet& g : graphs)
        if (g.maxit == maxit && g.precise == want_precise && g.fwd == (int)fwd64() && g.restart == restart_max)
          cached = &g;
    auto capture = [&](cudaStream_t cs, int which, int order, cudaGraphExec_t* out) -> cudaError_t {
      cudaGraph_t graph = nullptr;
      if (which >= 0) use(sub[which]);
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      if (order == 0) {
        enqueue_front(cs, maxit);
        enqueue_back(cs);
      } else {
        enqueue_back(cs);
        enqueue_front(cs, maxit);
      }
      e = cudaStreamEndCapture(cs, &graph);
      use(full);
      if (e != cudaSuccess) return e;
      size_t nn = 0;
      if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess) (which == 1 ? nodes2 : nodes1) = (long long)nn;
      e = cudaGraphInstantiate(out, graph, 0);
      cudaGraphDestroy(graph);
      return e;
    };
    if (split) {
      // the second half starts with its front part, then iterates
      // back + front: half an iteration behind the first half
      CK(cudaEventRecord(ev_fork, st));
      CK(cudaStreamWaitEvent(st2, ev_fork, 0));
      use(sub[1]);
      enqueue_front(st2, maxit);
      use(full);
    }
    cudaGraphExec_t pexec = nullptr, pexec2 = nullptr;
    if (cached) {
      exec = cached->exec;
      exec2 = cached->exec2;
      pexec = cached->pexec;
      pexec2 = cached->pexec2;
      nodes1 = cached->nodes1;
      nodes2 = cached->nodes2;
    } else if (!split) {
      ce = capture(st, -1, 0, &exec);
    } else {
      ce = capture(st, 0, 0, &exec);
      if (ce == cudaSuccess) ce = capture(st2, 1, 1, &exec2);
    }
    // the same iteration with the precise H X' (captured up front; the node
    // counts are equal)
    if (!cached && ce == cudaSuccess && want_precise) {
      hx64 = true;
      const long long n1 = nodes1, n2 = nodes2;
      ce = split ? capture(st, 0, 0, &pexec) : capture(st, -1, 0, &pexec);
      if (ce == cudaSuccess && split) ce = capture(st2, 1, 1, &pexec2);
      nodes1 = n1;
      nodes2 = n2;
      hx64 = false;
    }
    bool precise = false;
    if (trace_) {
      cudaStreamSynchronize(st);
      if (split) cudaStreamSynchronize(st2);
      std::fprintf(stderr, "[dgdft] run: graphs captured at %.2f ms\n", trace_ms());
    }
    if (ce != cudaSuccess) {
      if (exec) cudaGraphExecDestroy(exec);
      if (exec2) cudaGraphExecDestroy(exec2);
      if (pexec) cudaGraphExecDestroy(pexec);
      if (pexec2) cudaGraphExecDestroy(pexec2);
      if (split) {
        cudaEventRecord(ev_join, st2);
        cudaStreamWaitEvent(st, ev_join, 0);
      }
      return ctx->fail(DGDFT_ECUDA, "graph capture: " + cuda_err_string(ce));
    }
    if (!cached && cacheable) {
      GraphSet g;
      g.maxit = maxit;
      g.precise = want_precise;
      g.fwd = (int)fwd64();
      g.restart = restart_max;
      g.exec = exec;
      g.exec2 = exec2;
      g.pexec = pexec;
      g.pexec2 = pexec2;
      g.nodes1 = nodes1;
      g.nodes2 = nodes2;
      graphs.push_back(g);
      cached = &graphs.back();
    }
    const int nel = (int)ids.size();
    const int every = std::max(1, ctx->cfg.check_every);
    std::vector<std::vector<double>> hist(nel);
    std::vector<int> seen_restarts(nel, 0);
    std::vector<double> resbuf;
    int launched = 0;
    dgdft_status rs = DGDFT_OK;
    int since_refresh = 0;
    while (launched <= maxit + 1) {
      if (refresh_every > 0 && !split && since_refresh >= refresh_every) {
        // recompute HX = H X: the updates HX <- [HX HW HP] Y accumulate
        // rounding in the working precision
        launch_apply_h<real>(batch, bref<real>(BX), bref<real>(BHX), 0, st, fwd64());
        since_refresh = 0;
      }
      for (int k = 0; k < every && launched <= maxit + 1; ++k, ++launched, ++since_refresh) {
        ce = cudaGraphLaunch(precise ? pexec : exec, st);
        if (ce == cudaSuccess && split) ce = cudaGraphLaunch(precise ? pexec2 : exec2, st2);
        if (ce != cudaSuccess) break;
        graph_kernels += nodes1 + (split ? nodes2 : 0);
      }
      if (ce != cudaSuccess) break;
      if (split) {
        ce = cudaStreamSynchronize(st2);
        if (ce != cudaSuccess) break;
      }
      if ((rs = read_states()) != DGDFT_OK) break;
      if (trace_) {
        // diagnostic trace of element 0 (DGDFT_TRACE set in the environment)
        std::vector<double> r0(h[0].J);
        if (ctx_copy(ctx, r0.data(), h[0].res, sizeof(double) * h[0].J, cudaMemcpyDeviceToHost) == cudaSuccess)
          std::fprintf(stderr, "[dgdft] %s it=%d active=%d max_res=%.3e\n", sizeof(real) == 4 ? "fp32" : "fp64",
                       h_state[ST_ITER], h_state[ST_ACTIVE], *std::max_element(r0.begin(), r0.end()));
      }
      bool any = false;
      std::vector<double> active_res;  // read only with a stall window
      for (int i = 0; i < nel; ++i) {
        int* sw = &h_state[(size_t)i * STATE_WORDS];
        if (!sw[ST_ACTIVE]) continue;
        any = true;
        if (stall_window > 0) {
          if (sw[ST_NRESTART] != seen_restarts[i]) {
            // restarted since the last poll: the perturbed block climbs back
            // from a higher residual, which is not a stall
            seen_restarts[i] = sw[ST_NRESTART];
            hist[i].clear();
          }
          resbuf.resize(h[i].J);
          ce = ctx_copy(ctx, resbuf.data(), h[i].res, sizeof(double) * h[i].J, cudaMemcpyDeviceToHost);
          if (ce != cudaSuccess) break;
          const double mx = *std::max_element(resbuf.begin(), resbuf.end());
          hist[i].push_back(mx);
          active_res.push_back(mx);
          const size_t L = hist[i].size();
          // stalled: the best residual of the last `stall_window` polls is not
          // stall_gain below the best one before them (the FP32 floor has
          // been reached).  Only near the floor (below max(10 tol, 1e-5)):
          // above it, up to max(100 tol, 1e-4), a plateau has to last four
          // times as long, since an element that leaves early at 2e-5 costs
          // ~10 more FP64 iterations while its FP32 iterations are free as
          // long as other elements still iterate; early plateaus of a random
          // start are never stalls.
          bool stalled = false, near_floor = false, stalled_any = false;
          auto stall_over = [&](size_t win) {
            if (hist[i].size() <= win) return false;
            const double before = *std::min_element(hist[i].begin(), hist[i].end() - win);
            const double recent = *std::min_element(hist[i].end() - win, hist[i].end());
            return recent > stall_gain * before;
          };
          if (L > (size_t)stall_window) {
            const double recent = *std::min_element(hist[i].end() - stall_window, hist[i].end());
            stalled_any = stall_over((size_t)stall_window);  // the learned network's fallback
            if (recent < std::max(10.0 * tol, 1e-5)) {
              stalled = stall_over((size_t)stall_window);
              near_floor = true;
            } else if (recent < std::max(100.0 * tol, 1e-4)) {
              stalled = stall_over(4 * (size_t)stall_window);
              near_floor = true;
            }
          }
          if (stalled_any && learned && !sw[ST_TETER]) {
            // the learned preconditioner stalled: fall back to Teter
            int one = 1;
            ce = ctx_copy(ctx, h[i].state + ST_TETER, &one, sizeof(int), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) break;
            int fb = sw[ST_FALLBACK] + 1;
            ce = ctx_copy(ctx, h[i].state + ST_FALLBACK, &fb, sizeof(int), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) break;
            hist[i].clear();
          } else if (stalled && near_floor) {
            int zero = 0;
            ce = ctx_copy(ctx, h[i].state + ST_ACTIVE, &zero, sizeof(int), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) break;
          }
        }
      }
      if (ce != cudaSuccess || !any) break;
      if (pexec && !precise && !active_res.empty()) {
        // switch once the median active element is below the threshold: the
        // rest would otherwise stall at the FP32 floor before a laggard
        // catches up
        std::nth_element(active_res.begin(), active_res.begin() + active_res.size() / 2, active_res.end());
        if (active_res[active_res.size() / 2] < precise_below) precise = true;
      }
    }
    if (!cached) {
      cudaGraphExecDestroy(exec);
      if (exec2) cudaGraphExecDestroy(exec2);
      if (pexec) cudaGraphExecDestroy(pexec);
      if (pexec2) cudaGraphExecDestroy(pexec2);
    }
    if (split) {
      // later work on the caller's stream sees the second half's results
      cudaEventRecord(ev_join, st2);
      cudaStreamWaitEvent(st, ev_join, 0);
    }
    if (ce != cudaSuccess) return ctx->fail(DGDFT_ECUDA, "LOBPCG iteration: " + cuda_err_string(ce));
    if (rs != DGDFT_OK) return rs;
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (res_out) {
      res_out->clear();
      for (int i = 0; i < nel; ++i) {
        std::vector<double> r(h[i].m);
        CK(ctx_copy(ctx, r.data(), h[i].res, sizeof(double) * h[i].m, cudaMemcpyDeviceToHost));
        res_out->insert(res_out->end(), r.begin(), r.end());
      }
    }
    return read_states();
  }

  const real* current_x(int i) const {
    return h[i].blk[BX][h_state[(size_t)i * STATE_WORDS + ST_PARITY] & 1];
  }
};

// Seeded standard-normal default initial block (splitmix64 + Box-Muller).
void default_x0(std::vector<double>& x, int elem) {
  uint64_t s = 0x9E3779B97F4A7C15ull * (uint64_t)(elem + 1);
  auto next = [&]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (size_t i = 0; i < x.size(); i += 2) {
    const double u1 = next(), u2 = next();
    const double r = std::sqrt(-2.0 * std::log(u1));
    x[i] = r * std::cos(2.0 * M_PI * u2);
    if (i + 1 < x.size()) x[i + 1] = r * std::sin(2.0 * M_PI * u2);
  }
}

// FP64 restriction + orthonormalisation (Sec. II.A; Eq. orthonormal) of the
// blocks xs[q] of wave elements idx[q] into out[q]: Phi~ = the first K[q]
// columns of X restricted to E_K; G = Phi~^T Phi~; the lowest J[q]
// eigenpairs of the pencil I y = th G y (th = 1 / sigma^2: the largest
// singular values) give Y1 with Y1^T G Y1 = I, U = Phi~ Y1 (those left
// singular vectors up to rotation); one more pass on U restores
// orthonormality to rounding; scaled by 1/sqrt(dV).  K = J is the paper's
// procedure (all J restricted vectors kept); K = m restricts all computed
// vectors and keeps the top J.  Everything is enqueued on the context's stream with one
// scratch allocation and one synchronisation for all listed elements;
// rank_ok[q] is false where the restricted block is rank deficient.
dgdft_status orthonormalise(dgdft_alb_ctx* ctx, Wave<double>& w, const std::vector<int>& idx,
                            const std::vector<const double*>& xs, const std::vector<int>& Js,
                            const std::vector<int>& Ks, const std::vector<double*>& out,
                            std::vector<char>& rank_ok) {
  cudaStream_t st = ctx->stream;
  const size_t nq = idx.size();
  rank_ok.assign(nq, 0);
  if (nq == 0) return DGDFT_OK;
  int Jmax = 1, Kmax = 1;
  size_t nemax = 1;
  for (size_t q = 0; q < nq; ++q) {
    Jmax = std::max(Jmax, Js[q]);
    Kmax = std::max(Kmax, Ks[q]);
    nemax = std::max(nemax, (size_t)ctx->el[w.ids[idx[q]]].ne());
  }
  const size_t jj = (size_t)Jmax * Jmax, kk = (size_t)Kmax * Kmax;
  // per element: phi_t (ne x K), U (ne x J), G (K x K), G2 (J x J), Y1
  // (K x J), Y2 (J x J), I (K x K), diag(1..J) (J x J), theta, Rayleigh-Ritz
  // work; then the task arrays, the Gram partials and the checks, so that
  // each phase is one launch over all elements
  const size_t per = nemax * Kmax + nemax * Jmax + 3 * kk + 3 * jj + Kmax + rr_work_doubles(Kmax, Kmax);
  const size_t npart = ortho_partial_doubles((int)nq, (int)nemax, Kmax);
  const size_t nbytes = sizeof(double) * (per * nq + nq + npart) + 2 * nq * sizeof(RRTask) +
                        4 * nq * sizeof(OrthoTask) + (10 * nq + 32) * ALIGN;
  if (nbytes > ctx->ortho_cap) {
    if (ctx->ortho_buf) cudaFree(ctx->ortho_buf);
    ctx->ortho_buf = nullptr;
    ctx->ortho_cap = 0;
    CK(cudaMalloc(&ctx->ortho_buf, nbytes));
    ctx->ortho_cap = nbytes;
  }
  Arena a;
  a.base = (char*)ctx->ortho_buf;
  a.cap = nbytes;
  struct Slot {
    double *phit, *U, *G, *G2, *Y1, *Y2, *mats, *th, *work;
  };
  std::vector<Slot> sl(nq);
  for (size_t q = 0; q < nq; ++q) {
    Slot& z = sl[q];
    z.phit = (double*)a.take(sizeof(double) * nemax * Kmax);
    z.U = (double*)a.take(sizeof(double) * nemax * Jmax);
    z.G = (double*)a.take(sizeof(double) * kk);
    z.G2 = (double*)a.take(sizeof(double) * jj);
    z.Y1 = (double*)a.take(sizeof(double) * kk);
    z.Y2 = (double*)a.take(sizeof(double) * jj);
    z.mats = (double*)a.take(sizeof(double) * (kk + jj));
    z.th = (double*)a.take(sizeof(double) * Kmax);
    z.work = (double*)a.take(sizeof(double) * rr_work_doubles(Kmax, Kmax));
  }
  double* chk = (double*)a.take(sizeof(double) * nq);
  double* part = (double*)a.take(sizeof(double) * npart);
  RRTask* dt = (RRTask*)a.take(2 * nq * sizeof(RRTask));  // [0, nq): first pass, [nq, 2nq): second
  // [0, nq): Gram of Phi~, then U = Phi~ Y1, Gram of U, out = U Y2
  OrthoTask* ot = (OrthoTask*)a.take(4 * nq * sizeof(OrthoTask));
  if (!chk || !dt || !ot || !part || !sl.back().work) return ctx->fail(DGDFT_ENOMEM, "orthonormalisation scratch");
  std::vector<double> hm((kk + jj) * nq, 0.0);
  std::vector<RRTask> ht(2 * nq);
  std::vector<OrthoTask> hot(4 * nq);
  for (size_t q = 0; q < nq; ++q) {
    const int J = Js[q], K = Ks[q], ne = ctx->el[w.ids[idx[q]]].ne();
    double* id = hm.data() + (kk + jj) * q;  // K x K identity
    double* dg = id + kk;                    // diag(1..J)
    for (int c = 0; c < K; ++c) id[c + (size_t)c * K] = 1.0;
    for (int c = 0; c < J; ++c) dg[c + (size_t)c * J] = 1.0 + c;
    for (int k = 0; k < 2; ++k) {
      const int n = k ? J : K;
      RRTask& t = ht[k * nq + q];
      t = RRTask{};
      t.A = sl[q].mats + (k ? kk : 0);
      t.B = k ? sl[q].G2 : sl[q].G;
      t.ld = n;
      t.mode = RR_FIXED;
      t.n_fixed = n;
      t.m = J;
      t.Y = k ? sl[q].Y2 : sl[q].Y1;
      t.ldy = n;
      t.theta = sl[q].th;
      t.work = sl[q].work;
      t.state = nullptr;
      t.cond_max = 1e30;
    }
    hot[q] = OrthoTask{sl[q].phit, nullptr, sl[q].G, ne, K, 0};
    hot[nq + q] = OrthoTask{sl[q].phit, sl[q].Y1, sl[q].U, ne, J, K};
    hot[2 * nq + q] = OrthoTask{sl[q].U, nullptr, sl[q].G2, ne, J, 0};
    hot[3 * nq + q] = OrthoTask{sl[q].U, sl[q].Y2, out[q], ne, J, 0};
    CK(cudaMemcpyAsync(sl[q].mats, id, sizeof(double) * (kk + jj), cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(dt, ht.data(), sizeof(RRTask) * ht.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ot, hot.data(), sizeof(OrthoTask) * hot.size(), cudaMemcpyHostToDevice, st));
  const int nqi = (int)nq, nem = (int)nemax;
  // Phi~ and G = Phi~^T Phi~ for every element, then one Rayleigh-Ritz launch
  for (size_t q = 0; q < nq; ++q) {
    const ElemHost& eh = ctx->el[w.ids[idx[q]]];
    const dgdft_element_desc& d = eh.d;
    launch_restrict<double>(xs[q], eh.ng(), d.nx, d.ny, d.e_lo, d.e_hi, Ks[q], sl[q].phit, st);
  }
  launch_ortho_gram(ot, nqi, nem, Kmax, part, st);
  launch_rr(dt, nqi, st, Kmax, Jmax);
  // U = Phi~ Y1 and its Gram, second Rayleigh-Ritz launch
  launch_ortho_apply(ot + nq, nqi, nem, Jmax, Kmax, st);
  launch_ortho_gram(ot + 2 * nq, nqi, nem, Jmax, part, st);
  launch_rr(dt + nq, nqi, st, Jmax, Jmax);
  launch_ortho_apply(ot + 3 * nq, nqi, nem, Jmax, Jmax, st);
  for (size_t q = 0; q < nq; ++q) {
    const ElemHost& eh = ctx->el[w.ids[idx[q]]];
    launch_scale(out[q], (size_t)eh.ne() * Js[q], 1.0 / std::sqrt(eh.dv()), st);
    CK(cudaMemcpyAsync(chk + q, sl[q].th, sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  std::vector<double> hchk(nq);
  CK(cudaMemcpyAsync(hchk.data(), chk, sizeof(double) * nq, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  for (size_t q = 0; q < nq; ++q) rank_ok[q] = std::isfinite(hchk[q]) ? 1 : 0;
  return DGDFT_OK;
}

dgdft_status alb_orthonormalise(dgdft_alb_ctx* ctx, Wave<double>& w, int i, const double* x, int J, int K,
                                double* phi_dev_out) {
  std::vector<char> ok;
  dgdft_status s = orthonormalise(ctx, w, {i}, {x}, {J}, {K}, {phi_dev_out}, ok);
  if (s != DGDFT_OK) return s;
  if (!ok[0]) return ctx->fail(DGDFT_ENOTCONV, "orthonormalisation: restricted block is rank deficient");
  return DGDFT_OK;
}

template <class real>
dgdft_status copy_block_to(Wave<real>& w, int i, Wave<double>& dst, int di, cudaStream_t st) {
  const ElemDev<real>& E = w.h[i];
  launch_convert<real, double>(w.current_x(i), dst.h[di].blk[BX][0], (size_t)E.ng * E.m, st);
  return DGDFT_OK;
}

dgdft_status finish_wave(dgdft_alb_ctx* ctx, Wave<double>& w, int wave_idx, double seconds,
                         const std::vector<int>& extra_iters, const std::vector<int>& extra_fb,
                         const std::vector<double>& bulk_res, long long graph_kernels,
                         const std::vector<int>& restarts, bool scf = false,
                         const std::vector<int>& bulk_err = std::vector<int>()) {
  const size_t nel = w.ids.size();
  std::vector<int> idx(nel), Js(nel), Ks(nel);
  std::vector<const double*> xs(nel);
  std::vector<double*> outs(nel);
  for (size_t i = 0; i < nel; ++i) {
    ElemHost& eh = ctx->el[w.ids[i]];
    const int J = w.h[i].J, ne = eh.ne();
    if (!eh.d_phi) {
      CK(cudaMalloc(&eh.d_phi, sizeof(double) * (size_t)ne * J));
      CK(cudaMalloc(&eh.d_eig, sizeof(double) * J));
      CK(cudaMalloc(&eh.d_res, sizeof(double) * J));
    }
    idx[i] = (int)i;
    Js[i] = J;
    Ks[i] = ctx->cfg.restrict_all ? w.h[i].m : J;
    xs[i] = w.current_x((int)i);
    outs[i] = eh.d_phi;
    CK(cudaMemcpyAsync(eh.d_eig, w.h[i].theta, sizeof(double) * J, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(eh.d_res, w.h[i].res, sizeof(double) * J, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  std::vector<char> rank_ok;
  {
    dgdft_status so = orthonormalise(ctx, w, idx, xs, Js, Ks, outs, rank_ok);
    if (so != DGDFT_OK) return so;
  }
  // eigenvalues and residuals of every element to the host, one wait
  for (size_t i = 0; i < nel; ++i) {
    ElemHost& eh = ctx->el[w.ids[i]];
    const ElemDev<double>& E = w.h[i];
    eh.eig.resize(E.J);
    eh.resid.resize(E.J);
    CK(cudaMemcpyAsync(eh.eig.data(), E.theta, sizeof(double) * E.J, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(eh.resid.data(), E.res, sizeof(double) * E.J, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < nel; ++i) {
    ElemHost& eh = ctx->el[w.ids[i]];
    const ElemDev<double>& E = w.h[i];
    const int* sw = &w.h_state[i * STATE_WORDS];
    const int m = E.m;
    const double* x = xs[i];
    const dgdft_status s = rank_ok[i] ? DGDFT_OK : DGDFT_ENOTCONV;
    if (ctx->cfg.keep_block) {
      eh.block.resize((size_t)eh.ng() * m);
      CK(ctx_copy(ctx, eh.block.data(), x, sizeof(double) * eh.block.size(), cudaMemcpyDeviceToHost));
    } else {
      eh.block.clear();
    }
    double mx = 0.0;
    for (double r : eh.resid) mx = std::max(mx, r);
    // (an SCF step's FP64 stage is only the residual check, whose pass counts
    // as one in the FP64 wave's iteration word)
    eh.rep.iterations = (scf && !extra_iters.empty()) ? extra_iters[i]
                                                      : sw[ST_ITER] + (extra_iters.empty() ? 0 : extra_iters[i]);
    eh.rep.fallbacks = sw[ST_FALLBACK] + (extra_fb.empty() ? 0 : extra_fb[i]);
    eh.rep.iterations_bulk = extra_iters.empty() ? 0 : extra_iters[i];
    eh.rep.resid_bulk = bulk_res.empty() ? 0.0 : bulk_res[i];
    eh.rep.max_resid = mx;
    eh.rep.wave = wave_idx;
    eh.rep.seconds = seconds;
    eh.rep.graph_kernels = graph_kernels;
    eh.rep.restarts = restarts.empty() ? 0 : restarts[i];
    // an SCF step has no tolerance: OK unless the element failed.  A
    // bounded device wait that ran out (in either stage) is reported as such
    // even when the FP64 stage went on to converge the element.
    const int err = sw[ST_ERROR] | (bulk_err.empty() ? 0 : bulk_err[i]);
    eh.rep.status = (err & ERR_TIMEOUT)                   ? DGDFT_ETIMEOUT
                    : (sw[ST_ERROR] != 0 || s != DGDFT_OK) ? DGDFT_ENOTCONV
                    : (scf || mx <= ctx->cfg.tol)          ? DGDFT_OK
                                                           : DGDFT_ENOTCONV;
    eh.solved = true;
  }
  return DGDFT_OK;
}

// The waves of one solve: FP32 bulk stage (mixed form only) and FP64 stage.
struct WavePair {
  std::unique_ptr<Wave<float>> w32;
  std::unique_ptr<Wave<double>> w64;
};
void free_wave_pair(void* p) { delete static_cast<WavePair*>(p); }

// The FP32 and FP64 waves of `ids`: the resident pair when keep and one is
// cached, else a new pair (cached when keep).
dgdft_status get_waves(dgdft_alb_ctx* ctx, const std::vector<int>& ids, bool keep, WavePair*& wp,
                       std::unique_ptr<WavePair>& owned) {
  const dgdft_alb_config& c = ctx->cfg;
  const bool mixed = c.precision == DGDFT_PREC_MIXED;
  if (keep && ctx->cache) {
    wp = static_cast<WavePair*>(ctx->cache);
  } else {
    owned.reset(new WavePair());
    wp = owned.get();
    dgdft_status s;
    if (mixed) {
      wp->w32.reset(new Wave<float>());
      // Cholesky condition limit of the FP32 stage's pencil: the Gram
      // products (compensated SIMT ~2e-7 relative; TF32 split ~2^-22 per
      // product) tolerate nearly dependent [X W P] up to 1e6
      const double cond32 = 1e6;
      // an element whose pencil fails at every level is restarted (X
      // perturbed, P dropped) up to 8 times before it is left to the FP64 stage
      if ((s = wp->w32->build(ctx, ids, cond32, 8)) != DGDFT_OK) return s;
    }
    wp->w64.reset(new Wave<double>());
    if ((s = wp->w64->build(ctx, ids, 1e14)) != DGDFT_OK) return s;
    if (keep) {
      ctx->drop_cache();
      ctx->cache = owned.release();
      ctx->cache_free = free_wave_pair;
      ctx->cache_proj_version.clear();
      for (const ElemHost& eh : ctx->el) ctx->cache_proj_version.push_back(eh.proj_version);
    }
  }
  return DGDFT_OK;
}

dgdft_status solve_wave(dgdft_alb_ctx* ctx, const std::vector<int>& ids, int wave_idx, bool keep) {
  auto t0 = std::chrono::steady_clock::now();
  const dgdft_alb_config& c = ctx->cfg;
  const bool mixed = c.precision == DGDFT_PREC_MIXED;
  WavePair* wp = nullptr;
  std::unique_ptr<WavePair> owned;
  {
    dgdft_status s = get_waves(ctx, ids, keep, wp, owned);
    if (s != DGDFT_OK) return s;
  }
  Wave<double>& w64 = *wp->w64;
  w64.graph_kernels = 0;
  if (wp->w32) wp->w32->graph_kernels = 0;
  std::vector<int> it32, fb32, rs32, er32;
  std::vector<double> res32;
  dgdft_status s;
  if (mixed) {
    Wave<float>& w32 = *wp->w32;
    if ((s = w32.load_inputs()) != DGDFT_OK) return s;
    // stage 1: FP32 storage and arithmetic, FP64 Rayleigh-Ritz.  It aims
    // below tol and ends an element when its residual stops improving: the
    // FP32 H apply leaves a floor near 2e-6 Ha (FFT rounding amplified by
    // |G|^2/2), from which FP64 needs two or three iterations
    const double tol1 = 0.6 * c.tol;
    std::vector<double> r32;
    const double precise_below = c.h_fp64_forward == 2 ? 1e-5 : 0.0;
    // hand over after two polls (8 iterations) without a 10% gain: measured
    // on the 36-element workload, waiting longer near the floor costs more
    // FP32 iterations than the extra FP64 iteration it saves
    if ((s = w32.run(tol1, c.maxit, 2, &r32, 0, false, precise_below, 0.9)) != DGDFT_OK) return s;
    {
      size_t off = 0;
      for (size_t i = 0; i < ids.size(); ++i) {
        const int m = w32.h[i].m, J = w32.h[i].J;
        res32.push_back(*std::max_element(r32.begin() + off, r32.begin() + off + J));
        off += m;
      }
    }
    // FP64 check from the FP32 Ritz block; LOBPCG continues in FP64 only for
    // the elements that miss tol
    for (size_t i = 0; i < ids.size(); ++i) {
      ElemHost& eh = ctx->el[ids[i]];
      launch_convert<double, double>(eh.d_veff, const_cast<double*>(w64.h[i].V), (size_t)eh.ng(), ctx->stream);
      copy_block_to<float>(w32, (int)i, w64, (int)i, ctx->stream);
      it32.push_back(w32.h_state[i * STATE_WORDS + ST_ITER]);
      fb32.push_back(w32.h_state[i * STATE_WORDS + ST_FALLBACK]);
      rs32.push_back(w32.h_state[i * STATE_WORDS + ST_NRESTART]);
      er32.push_back(w32.h_state[i * STATE_WORDS + ST_ERROR]);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (std::getenv("DGDFT_TRACE")) {
      for (size_t i = 0; i < ids.size(); ++i) {
        const int* sw = &w32.h_state[i * STATE_WORDS];
        if (sw[ST_ERROR] || sw[ST_ITER] < 50 || sw[ST_NRESTART])
          std::fprintf(stderr, "[dgdft] fp32 element %zu: iter %d err %d fallback %d restarts %d converged %d\n", i,
                       sw[ST_ITER], sw[ST_ERROR], sw[ST_FALLBACK], sw[ST_NRESTART], sw[ST_CONVERGED]);
      }
    }
    auto t1 = std::chrono::steady_clock::now();
    if ((s = w64.verify(c.tol)) != DGDFT_OK) return s;
    bool all = true;
    int nconv = 0;
    for (size_t i = 0; i < ids.size(); ++i) {
      all = all && w64.h_state[i * STATE_WORDS + ST_CONVERGED];
      nconv += w64.h_state[i * STATE_WORDS + ST_CONVERGED] != 0;
    }
    auto t2 = std::chrono::steady_clock::now();
    if (!all && (s = w64.run(c.tol, c.maxit, 0, nullptr, 0, true)) != DGDFT_OK) return s;
    if (std::getenv("DGDFT_TRACE")) {
      CK(cudaStreamSynchronize(ctx->stream));
      auto t3 = std::chrono::steady_clock::now();
      std::fprintf(stderr, "[dgdft] fp32 stage %.3f s, verify %.3f s (%d/%zu pass), fp64 stage %.3f s\n",
                   std::chrono::duration<double>(t1 - t0).count(), std::chrono::duration<double>(t2 - t1).count(),
                   nconv, ids.size(), std::chrono::duration<double>(t3 - t2).count());
    }
  } else {
    if ((s = w64.load_inputs()) != DGDFT_OK) return s;
    if ((s = w64.run(c.tol, c.maxit, 0, nullptr)) != DGDFT_OK) return s;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const long long gk = w64.graph_kernels + (wp->w32 ? wp->w32->graph_kernels : 0);
  return finish_wave(ctx, w64, wave_idx, secs, it32, fb32, res32, gk, rs32, false, er32);
}

// One SCF step for a resident single-wave workload (Sec. II.B: in every SCF
// iteration the ALBs are refined by a few LOBPCG iterations that start from
// those of the previous SCF step, under the updated potential).  Each element
// starts from the block given by set_initial since the last solve or step,
// else from its resident block of the previous solve or step; exactly n_iter
// iterations run in the context's precision (FP32 in the mixed form), with no
// tolerance, then the FP64 residual check, restriction and orthonormalisation.
dgdft_status scf_wave(dgdft_alb_ctx* ctx, const std::vector<int>& ids, int n_iter) {
  auto t0 = std::chrono::steady_clock::now();
  const bool mixed = ctx->cfg.precision == DGDFT_PREC_MIXED;
  WavePair* resident = static_cast<WavePair*>(ctx->cache);
  std::vector<const double*> warm(ids.size(), nullptr);
  for (size_t i = 0; i < ids.size(); ++i) {
    const ElemHost& eh = ctx->el[ids[i]];
    // a resident wave pair was made by a solve or step over every element
    if (eh.x0_fresh) warm[i] = eh.d_x0;
    else if (resident) warm[i] = resident->w64->current_x((int)i);
    else return ctx->fail(DGDFT_ESTATE, "SCF step: no block to start from (solve first, or set_initial)");
  }
  WavePair* wp = nullptr;
  std::unique_ptr<WavePair> owned;
  dgdft_status s = get_waves(ctx, ids, true, wp, owned);
  if (s != DGDFT_OK) return s;
  Wave<double>& w64 = *wp->w64;
  w64.graph_kernels = 0;
  std::vector<int> it32, fb32, rs32, er32;
  std::vector<double> res32;
  const bool trace = std::getenv("DGDFT_TRACE") != nullptr;
  auto stamp = [&](const char* what) {
    if (!trace) return;
    cudaStreamSynchronize(ctx->stream);
    std::fprintf(stderr, "[dgdft] scf step: %s at %.2f ms\n", what,
                 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  };
  stamp("waves ready");
  if (n_iter == 0) {
    // no iteration: Rayleigh-Ritz of the starting block and its FP64
    // residuals under the current potential
    if ((s = w64.load_inputs(&warm)) != DGDFT_OK) return s;
    if ((s = w64.run(0.0, 0, 0, nullptr)) != DGDFT_OK) return s;
  } else if (mixed) {
    Wave<float>& w32 = *wp->w32;
    w32.graph_kernels = 0;
    if ((s = w32.load_inputs(&warm)) != DGDFT_OK) return s;
    stamp("inputs converted");
    std::vector<double> r32;
    if ((s = w32.run(0.0, n_iter, 0, &r32)) != DGDFT_OK) return s;
    stamp("FP32 iterations done");
    size_t off = 0;
    for (size_t i = 0; i < ids.size(); ++i) {
      ElemHost& eh = ctx->el[ids[i]];
      const int m = w32.h[i].m, J = w32.h[i].J;
      res32.push_back(*std::max_element(r32.begin() + off, r32.begin() + off + J));
      off += m;
      launch_convert<double, double>(eh.d_veff, const_cast<double*>(w64.h[i].V), (size_t)eh.ng(), ctx->stream);
      copy_block_to<float>(w32, (int)i, w64, (int)i, ctx->stream);
      it32.push_back(w32.h_state[i * STATE_WORDS + ST_ITER]);
      fb32.push_back(w32.h_state[i * STATE_WORDS + ST_FALLBACK]);
      rs32.push_back(w32.h_state[i * STATE_WORDS + ST_NRESTART]);
      er32.push_back(w32.h_state[i * STATE_WORDS + ST_ERROR]);
    }
    if ((s = w64.verify(ctx->cfg.tol)) != DGDFT_OK) return s;
    stamp("FP64 check done");
  } else {
    if ((s = w64.load_inputs(&warm)) != DGDFT_OK) return s;
    if ((s = w64.run(0.0, n_iter, 0, nullptr)) != DGDFT_OK) return s;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const long long gk = w64.graph_kernels + (wp->w32 ? wp->w32->graph_kernels : 0);
  s = finish_wave(ctx, w64, 0, secs, it32, fb32, res32, gk, rs32, true, er32);
  stamp("restriction and orthonormalisation done");
  return s;
}

// Device-memory admission: elements in order, greedily into waves that fit
// the budget (each element with its share of the wave-level buffers).
dgdft_status plan_waves(dgdft_alb_ctx* ctx, std::vector<std::vector<int>>& waves) {
  size_t cap = ctx->cfg.hbm_cap_bytes;
  if (cap == 0) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    cap = (size_t)(0.9 * (double)fr);
  }
  size_t acc = 0;
  for (int id = 0; id < (int)ctx->el.size(); ++id) {
    const ElemHost& eh = ctx->el[id];
    if (!eh.has_v) return ctx->fail(DGDFT_ESTATE, "element without potential");
    // plus the element's share of the wave-level buffers (Gram partials and
    // residual partial sums, sized here by the element itself)
    const size_t m = (size_t)eh.d.n_compute, ng = (size_t)eh.ng();
    const size_t shared = sizeof(double) * (((ng + 2047) / 2048) * 12 * ((m + 63) / 64) * ((m + 63) / 64) * 4096 +
                                            m * (size_t)nchunk_rows((int)ng) * 4);
    size_t b = elem_bytes<double>(eh) + shared;
    if (ctx->cfg.precision == DGDFT_PREC_MIXED) b += elem_bytes<float>(eh) + shared;
    if (b > cap) return ctx->fail(DGDFT_ENOMEM, "one element exceeds the device-memory budget");
    if (waves.empty() || acc + b > cap) {
      waves.emplace_back();
      acc = 0;
    }
    waves.back().push_back(id);
    acc += b;
  }
  // a single wave stays resident for later solves unless projectors changed
  if (waves.size() != 1) ctx->drop_cache();
  if (waves.size() == 1 && ctx->cache) {
    bool same = ctx->cache_proj_version.size() == ctx->el.size();
    for (size_t i = 0; same && i < ctx->el.size(); ++i) same = ctx->cache_proj_version[i] == ctx->el[i].proj_version;
    if (!same) ctx->drop_cache();
  }
  return DGDFT_OK;
}

}  // namespace

// ------------------------------------------------------------------ C-ABI

extern "C" {

void dgdft_alb_config_init(dgdft_alb_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = DGDFT_PREC_FP64;
  cfg->precond = DGDFT_PRECOND_TETER;
  cfg->tol = 1e-6;
  cfg->maxit = 400;
  cfg->check_every = 4;
  cfg->hbm_cap_bytes = 0;
  cfg->cuda_stream = nullptr;
  cfg->device = -1;
  cfg->keep_block = 0;
}

dgdft_status dgdft_alb_create(const dgdft_alb_config* cfg, int n_elem, const dgdft_element_desc* elems,
                              dgdft_alb_ctx** out) {
  if (!out) return DGDFT_EINVAL;
  *out = nullptr;
  if (!cfg || n_elem <= 0 || !elems) return DGDFT_EINVAL;
  if (cfg->precision != DGDFT_PREC_FP64 && cfg->precision != DGDFT_PREC_MIXED) return DGDFT_EINVAL;
  if (cfg->precond != DGDFT_PRECOND_TETER && cfg->precond != DGDFT_PRECOND_LEARNED) return DGDFT_EINVAL;
  if (!(cfg->tol > 0.0) || cfg->maxit <= 0) return DGDFT_EINVAL;
  if (cfg->bulk_kernels < 0 || cfg->bulk_kernels > 2) return DGDFT_EINVAL;
  if (cfg->restrict_all != 0 && cfg->restrict_all != 1) return DGDFT_EINVAL;
  if (!(cfg->ecut >= 0.0) || !std::isfinite(cfg->ecut)) return DGDFT_EINVAL;
  if (cfg->ecut > 0.0 && cfg->precond != DGDFT_PRECOND_TETER) return DGDFT_EINVAL;
  for (int i = 0; i < n_elem; ++i) {
    const dgdft_element_desc& d = elems[i];
    FftPlan p;
    if (d.nx < 4 || d.nx % 2 || !plan_length(d.nx / 2, p) || !plan_length(d.ny, p) || !plan_length(d.nz, p))
      return DGDFT_EINVAL;
    // one FP64 half-spectrum plane (two buffers) and one z-column tile must
    // fit a CTA's shared memory
    if ((long long)(d.nx / 2 + 1) * d.ny > 7000 || d.nz > 400) return DGDFT_EINVAL;
    if (!(d.Lx > 0 && d.Ly > 0 && d.Lz > 0)) return DGDFT_EINVAL;
    if (d.n_keep <= 0 || d.n_keep > d.n_compute) return DGDFT_EINVAL;
    const long long ng = (long long)d.nx * d.ny * d.nz;
    if (ng > (1ll << 30) || 3ll * d.n_compute > ng) return DGDFT_EINVAL;
    const int n3[3] = {d.nx, d.ny, d.nz};
    long long ne = 1;
    for (int a = 0; a < 3; ++a) {
      if (d.e_lo[a] < 0 || d.e_hi[a] > n3[a] || d.e_lo[a] >= d.e_hi[a]) return DGDFT_EINVAL;
      ne *= d.e_hi[a] - d.e_lo[a];
    }
    if (ne < d.n_keep) return DGDFT_EINVAL;
    // the LOBPCG basis [X W P] needs 3m independent planewaves in the set
    if (cfg->ecut > 0.0 && cutoff_set_size(d, cfg->ecut) < 3ll * d.n_compute) return DGDFT_EINVAL;
  }
  std::unique_ptr<dgdft_alb_ctx> ctx(new dgdft_alb_ctx());
  ctx->cfg = *cfg;
  // the caller's strings need not outlive the call
  if (cfg->autotune_cache) ctx->tune_path = cfg->autotune_cache;
  ctx->cfg.autotune_cache = nullptr;
  if (ctx->cfg.check_every < 1) ctx->cfg.check_every = 1;
  if (cfg->device_wait_polls < 0) return DGDFT_EINVAL;
  ctx->wait_polls = cfg->device_wait_polls;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return DGDFT_ECUDA;
  int dev = cfg->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return DGDFT_ECUDA;
  if (dev >= ndev || cudaSetDevice(dev) != cudaSuccess) return DGDFT_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DGDFT_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return DGDFT_ECUDA;
  ctx->device = dev;
  if (cfg->cuda_stream) {
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return DGDFT_ECUDA;
    ctx->own_stream = true;
  }
  init_hamiltonian_kernels();
  init_tf32_gram_kernel();
  init_tf32_update_kernel();
  init_rr_kernels();
  init_rr_df_kernel();
  init_blas_kernels();
  cudaGetLastError();  // attribute queries above must not leave an error behind
  ctx->el.resize(n_elem);
  for (int i = 0; i < n_elem; ++i) ctx->el[i].d = elems[i];
  if (cfg->precond_weights) {
    ctx->net = new ConvNet();
    std::string e = ctx->net->init(0, ctx->stream);
    if (e.empty()) e = ctx->net->load_file(cfg->precond_weights, ctx->stream);
    if (!e.empty()) {
      dgdft_alb_destroy(ctx.release());
      return DGDFT_EINVAL;
    }
  }
  *out = ctx.release();
  return DGDFT_OK;
}

// Copy n doubles into a resident device buffer (allocated on first use),
// rejecting non-finite values.
static dgdft_status copy_resident(dgdft_alb_ctx* ctx, double*& dst, const double* src, size_t n, int on_device) {
  if (!on_device)
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(src[i])) return ctx->fail(DGDFT_EINVAL, "non-finite input value");
  CK(cudaSetDevice(ctx->device));
  if (!dst) {
    cudaError_t e = cudaMalloc(&dst, sizeof(double) * n);
    if (e != cudaSuccess) {
      dst = nullptr;
      return ctx->fail(DGDFT_ENOMEM, "resident input allocation: " + cuda_err_string(e));
    }
  }
  CK(ctx_copy(ctx, dst, src, sizeof(double) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  if (on_device) {
    int* flag = nullptr;
    CK(cudaMalloc(&flag, sizeof(int)));
    int h = 0;
    cudaError_t e = ctx_copy(ctx, flag, &h, sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      launch_nonfinite(dst, n, flag, ctx->stream);
      e = ctx_copy(ctx, &h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    }
    cudaFree(flag);
    if (e != cudaSuccess) return ctx->fail(DGDFT_ECUDA, "input check: " + cuda_err_string(e));
    if (h) return ctx->fail(DGDFT_EINVAL, "non-finite input value");
  }
  return DGDFT_OK;
}

dgdft_status dgdft_alb_set_potential(dgdft_alb_ctx* ctx, int elem, const double* veff, int on_device) {
  if (!ctx || !veff || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  dgdft_status s = copy_resident(ctx, eh.d_veff, veff, (size_t)eh.ng(), on_device);
  eh.has_v = (s == DGDFT_OK);
  eh.solved = false;
  return s;
}

dgdft_status dgdft_alb_set_projectors(dgdft_alb_ctx* ctx, int elem, int n_proj, const int64_t* row_ptr,
                                      const int32_t* grid_idx, const double* val, const double* gamma) {
  if (!ctx || elem < 0 || elem >= (int)ctx->el.size() || n_proj < 0) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  if (n_proj == 0) {
    eh.prow.assign(1, 0);
    eh.pidx.clear();
    eh.pval.clear();
    eh.pgamma.clear();
    eh.proj_version += 1;
    return DGDFT_OK;
  }
  if (!row_ptr || !gamma) return DGDFT_EINVAL;
  if (row_ptr[0] != 0) return ctx->fail(DGDFT_EINVAL, "row_ptr[0] must be 0");
  for (int p = 0; p < n_proj; ++p)
    if (row_ptr[p + 1] < row_ptr[p]) return ctx->fail(DGDFT_EINVAL, "row_ptr not monotone");
  const int64_t nnz = row_ptr[n_proj];
  if (nnz > (1ll << 30) || (nnz > 0 && (!grid_idx || !val))) return DGDFT_EINVAL;
  const int ng = eh.ng();
  for (int64_t k = 0; k < nnz; ++k) {
    if (grid_idx[k] < 0 || grid_idx[k] >= ng) return ctx->fail(DGDFT_EINVAL, "projector index outside the grid");
    if (!std::isfinite(val[k])) return ctx->fail(DGDFT_EINVAL, "non-finite projector value");
  }
  for (int p = 0; p < n_proj; ++p)
    if (!std::isfinite(gamma[p])) return ctx->fail(DGDFT_EINVAL, "non-finite projector weight");
  // duplicate indices within one projector would double-count a point
  for (int p = 0; p < n_proj; ++p) {
    std::vector<int32_t> v(grid_idx + row_ptr[p], grid_idx + row_ptr[p + 1]);
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end())
      return ctx->fail(DGDFT_EINVAL, "duplicate grid index inside one projector");
  }
  eh.prow.assign(row_ptr, row_ptr + n_proj + 1);
  eh.pidx.assign(grid_idx, grid_idx + nnz);
  eh.pval.assign(val, val + nnz);
  eh.pgamma.assign(gamma, gamma + n_proj);
  eh.proj_version += 1;
  eh.solved = false;
  return DGDFT_OK;
}

dgdft_status dgdft_alb_set_initial(dgdft_alb_ctx* ctx, int elem, const double* x0, int on_device) {
  if (!ctx || !x0 || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  dgdft_status s = copy_resident(ctx, eh.d_x0, x0, (size_t)eh.ng() * eh.d.n_compute, on_device);
  eh.has_x0 = (s == DGDFT_OK);
  eh.x0_fresh = eh.has_x0;
  return s;
}

dgdft_status dgdft_alb_scf_step(dgdft_alb_ctx* ctx, int n_iter, dgdft_solve_report* per_elem) {
  if (!ctx || n_iter < 0) return DGDFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  std::vector<std::vector<int>> waves;
  dgdft_status s = plan_waves(ctx, waves);
  if (s != DGDFT_OK) return s;
  if (waves.size() != 1) return ctx->fail(DGDFT_ESTATE, "SCF steps need the workload resident in one wave");
  if ((s = scf_wave(ctx, waves[0], n_iter)) != DGDFT_OK) return s;
  for (ElemHost& eh : ctx->el) eh.x0_fresh = false;
  ctx->solved_any = true;
  dgdft_status out = DGDFT_OK;
  for (int i = 0; i < (int)ctx->el.size(); ++i) {
    if (per_elem) per_elem[i] = ctx->el[i].rep;
    if (ctx->el[i].rep.status == DGDFT_ETIMEOUT) out = DGDFT_ETIMEOUT;
    else if (ctx->el[i].rep.status != DGDFT_OK && out == DGDFT_OK) out = DGDFT_ENOTCONV;
  }
  if (out == DGDFT_ETIMEOUT) ctx->err = "a bounded device wait ran out";
  else if (out != DGDFT_OK) ctx->err = "some elements failed in the SCF step";
  return out;
}

dgdft_status dgdft_alb_solve(dgdft_alb_ctx* ctx, dgdft_solve_report* per_elem) {
  if (!ctx) return DGDFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  std::vector<std::vector<int>> waves;
  dgdft_status ps = plan_waves(ctx, waves);
  if (ps != DGDFT_OK) return ps;
  const bool keep = waves.size() == 1;
  for (size_t w = 0; w < waves.size(); ++w) {
    dgdft_status s = solve_wave(ctx, waves[w], (int)w, keep);
    if (s != DGDFT_OK) return s;
  }
  for (ElemHost& eh : ctx->el) eh.x0_fresh = false;
  ctx->solved_any = true;
  dgdft_status out = DGDFT_OK;
  for (int i = 0; i < (int)ctx->el.size(); ++i) {
    if (per_elem) per_elem[i] = ctx->el[i].rep;
    if (ctx->el[i].rep.status == DGDFT_ETIMEOUT) out = DGDFT_ETIMEOUT;
    else if (ctx->el[i].rep.status != DGDFT_OK && out == DGDFT_OK) out = DGDFT_ENOTCONV;
  }
  if (out == DGDFT_ETIMEOUT) ctx->err = "a bounded device wait ran out";
  else if (out != DGDFT_OK) ctx->err = "some elements did not reach the tolerance";
  return out;
}

dgdft_status dgdft_alb_get_basis(dgdft_alb_ctx* ctx, int elem, double* phi, double* eig, double* resid,
                                 int on_device) {
  if (!ctx || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  if (!eh.solved) return ctx->fail(DGDFT_ESTATE, "get_basis before solve");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t J = eh.d.n_keep;
  if (phi) CK(ctx_copy(ctx, phi, eh.d_phi, sizeof(double) * J * eh.ne(), k));
  if (eig) CK(ctx_copy(ctx, eig, eh.d_eig, sizeof(double) * J, k));
  if (resid) CK(ctx_copy(ctx, resid, eh.d_res, sizeof(double) * J, k));
  return DGDFT_OK;
}

const char* dgdft_alb_last_error(const dgdft_alb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void dgdft_alb_destroy(dgdft_alb_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  ctx->drop_cache();
  if (ctx->ortho_buf) cudaFree(ctx->ortho_buf);
  for (ElemHost& eh : ctx->el) eh.release();
  delete ctx->net;
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// ---------------------------------------------------------- step entry points

dgdft_status dgdft_alb_get_block(dgdft_alb_ctx* ctx, int elem, double* x, int on_device) {
  if (!ctx || !x || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  if (!eh.solved) return ctx->fail(DGDFT_ESTATE, "get_block before a solve");
  if (!eh.block.empty()) {
    if (on_device) {
      CK(ctx_copy(ctx, x, eh.block.data(), sizeof(double) * eh.block.size(), cudaMemcpyHostToDevice));
    } else {
      std::memcpy(x, eh.block.data(), sizeof(double) * eh.block.size());
    }
    return DGDFT_OK;
  }
  // no host copy: the FP64 wave of a single-wave workload stays resident
  // with the final block of the last solve or SCF step
  if (ctx->cache) {
    const WavePair* wp = static_cast<const WavePair*>(ctx->cache);
    const Wave<double>& w = *wp->w64;
    for (size_t i = 0; i < w.ids.size(); ++i) {
      if (w.ids[i] != elem) continue;
      const size_t n = (size_t)eh.ng() * eh.d.n_compute;
      CK(ctx_copy(ctx, x, w.current_x((int)i), sizeof(double) * n,
                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
      return DGDFT_OK;
    }
  }
  return ctx->fail(DGDFT_ESTATE, "no Ritz block: solve with keep_block, or keep the workload in one wave");
}

}  // extern "C"

namespace {

// A one-element wave in the context precision for step calls.
template <class real>
dgdft_status with_step_wave(dgdft_alb_ctx* ctx, int elem, Wave<real>& w) {
  if (elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (!ctx->el[elem].has_v) return ctx->fail(DGDFT_ESTATE, "element without potential");
  CK(cudaSetDevice(ctx->device));
  dgdft_status s = w.build(ctx, std::vector<int>{elem}, 1e14);
  if (s != DGDFT_OK) return s;
  if ((s = w.load_potential()) != DGDFT_OK) return s;
  return w.reset_states(ctx->cfg.tol);
}

template <class real>
dgdft_status step_in(dgdft_alb_ctx* ctx, real* dst, const double* src, size_t n, int on_device) {
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(double) * std::max<size_t>(n, 1)));
  cudaError_t e = ctx_copy(ctx, tmp, src, sizeof(double) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_convert<double, real>(tmp, dst, n, ctx->stream);
    e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return ctx->fail(DGDFT_ECUDA, "step input: " + cuda_err_string(e));
  return DGDFT_OK;
}

template <class real>
dgdft_status step_out(dgdft_alb_ctx* ctx, double* dst, const real* src, size_t n, int on_device) {
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(double) * std::max<size_t>(n, 1)));
  launch_convert<real, double>(src, tmp, n, ctx->stream);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess)
    e = ctx_copy(ctx, dst, tmp, sizeof(double) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (e != cudaSuccess) return ctx->fail(DGDFT_ECUDA, "step output: " + cuda_err_string(e));
  return DGDFT_OK;
}

template <class real>
dgdft_status apply_h_t(dgdft_alb_ctx* ctx, int elem, int k, const double* x, double* hx, int on_device) {
  Wave<real> w;
  dgdft_status s = with_step_wave<real>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  const size_t n = (size_t)w.h[0].ng * k;
  real* xs = w.h[0].blk[BW][0];
  real* ys = w.h[0].blk[BHW][0];
  if ((s = step_in<real>(ctx, xs, x, n, on_device)) != DGDFT_OK) return s;
  launch_apply_h<real>(w.batch, bptr<real>(xs), bptr<real>(ys), k, ctx->stream);
  CK(cudaGetLastError());
  return step_out<real>(ctx, hx, ys, n, on_device);
}

template <class real>
dgdft_status teter_t(dgdft_alb_ctx* ctx, int elem, int k, const double* r, const double* t_kin, double* wout,
                     int on_device) {
  Wave<real> w;
  dgdft_status s = with_step_wave<real>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  const size_t n = (size_t)w.h[0].ng * k;
  real* xs = w.h[0].blk[BW][0];
  real* ys = w.h[0].blk[BHW][0];
  if ((s = step_in<real>(ctx, xs, r, n, on_device)) != DGDFT_OK) return s;
  CK(ctx_copy(ctx, w.h[0].tkin, t_kin, sizeof(double) * k, cudaMemcpyHostToDevice));
  launch_teter<real>(w.batch, bptr<real>(xs), bptr<real>(ys), w.h[0].tkin, k, ctx->stream);
  CK(cudaGetLastError());
  return step_out<real>(ctx, wout, ys, n, on_device);
}

dgdft_status project_t(dgdft_alb_ctx* ctx, int elem, int k, const double* x, double* px, int on_device) {
  Wave<double> w;
  dgdft_status s = with_step_wave<double>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  const size_t n = (size_t)w.h[0].ng * k;
  double* xs = w.h[0].blk[BW][0];
  double* ys = w.h[0].blk[BHW][0];
  if ((s = step_in<double>(ctx, xs, x, n, on_device)) != DGDFT_OK) return s;
  launch_project(w.batch, bptr<double>(xs), bptr<double>(ys), k, ctx->stream);
  CK(cudaGetLastError());
  return step_out<double>(ctx, px, ys, n, on_device);
}

template <class real>
dgdft_status gram_t(dgdft_alb_ctx* ctx, int ng, int p, int q, const double* u, const double* v, double* c,
                    int on_device) {
  // a scratch wave-less batch: one ElemDev with only the state word set
  real *du = nullptr, *dv = nullptr;
  double *dc = nullptr, *part = nullptr;
  ElemDev<real>* de = nullptr;
  int* dstate = nullptr;
  const size_t tiles = ((p + 63) / 64) * ((q + 63) / 64);
  const size_t pcap = ((size_t)(ng + 2047) / 2048) * tiles * 4096;
  CK(cudaMalloc(&du, sizeof(real) * (size_t)ng * p));
  CK(cudaMalloc(&dv, sizeof(real) * (size_t)ng * q));
  CK(cudaMalloc(&dc, sizeof(double) * (size_t)p * q));
  CK(cudaMalloc(&part, sizeof(double) * pcap));
  CK(cudaMalloc(&de, sizeof(ElemDev<real>)));
  CK(cudaMalloc(&dstate, sizeof(int) * STATE_WORDS));
  dgdft_status s = step_in<real>(ctx, du, u, (size_t)ng * p, on_device);
  if (s == DGDFT_OK) s = step_in<real>(ctx, dv, v, (size_t)ng * q, on_device);
  if (s == DGDFT_OK) {
    ElemDev<real> E;
    std::memset(&E, 0, sizeof(E));
    E.m = std::max(p, q);
    E.ng = ng;
    E.state = dstate;
    int st[STATE_WORDS] = {0};
    st[ST_ACTIVE] = 1;
    ctx_copy(ctx, dstate, st, sizeof(st), cudaMemcpyHostToDevice);
    ctx_copy(ctx, de, &E, sizeof(E), cudaMemcpyHostToDevice);
    Batch<real> b;
    b.d_elems = de;
    b.s.nel = 1;
    b.s.max_m = E.m;
    b.s.max_ng = ng;
    GramJob<real> g;
    g.npairs = 1;
    g.a[0] = bptr<real>(du);
    g.b[0] = bptr<real>(dv);
    g.needs_p[0] = 0;
    g.out_id[0] = OUT_PTR;
    g.brow[0] = g.bcol[0] = 0;
    g.ncols_a = p;
    g.ncols_b = q;
    g.rows = ng;
    g.ld_in = ng;
    g.ld_out = p;
    g.out_ptr = dc;
    launch_gram<real>(b, g, part, pcap, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = ctx_copy(ctx, c, dc, sizeof(double) * (size_t)p * q, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = ctx->fail(DGDFT_ECUDA, "gram: " + cuda_err_string(e));
  }
  cudaFree(du);
  cudaFree(dv);
  cudaFree(dc);
  cudaFree(part);
  cudaFree(de);
  cudaFree(dstate);
  return s;
}

// The Gram products of one LOBPCG iteration on caller blocks, through the
// wave's own kernels (see dgdft_alb_lobpcg_gram).
template <class real>
dgdft_status lobpcg_gram_t(dgdft_alb_ctx* ctx, int elem, int has_p, const double* blocks, double* a, double* b,
                           double* xtw, int on_device) {
  // (a Wave<double> of a mixed context is its refinement stage: double-float)
  Wave<real> w;
  dgdft_status s = with_step_wave<real>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  ElemDev<real>& E = w.h[0];
  const int m = E.m;
  const size_t n = (size_t)E.ng * m;
  const int order[6] = {BX, BW, BP, BHX, BHW, BHP};
  for (int q = 0; q < 6; ++q)
    if ((s = step_in<real>(ctx, E.blk[order[q]][0], blocks + q * n, n, on_device)) != DGDFT_OK) return s;
  const int hp = has_p ? 1 : 0;
  CK(ctx_copy(ctx, E.state + ST_HAS_P, &hp, sizeof(int), cudaMemcpyHostToDevice));
  const size_t nn = (size_t)9 * m * m;
  CK(cudaMemsetAsync(E.gram, 0, sizeof(double) * 2 * nn, ctx->stream));
  CK(cudaMemsetAsync(E.gxw, 0, sizeof(double) * m * m, ctx->stream));
  w.gram_xtw(ctx->stream);
  w.gram_pencil(ctx->stream);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  int err = 0;
  CK(ctx_copy(ctx, &err, E.state + ST_ERROR, sizeof(int), cudaMemcpyDeviceToHost));
  if (err & ERR_TIMEOUT) return ctx->fail(DGDFT_ETIMEOUT, "lobpcg_gram: a bounded device wait ran out");
  std::vector<double> g(2 * nn);
  CK(ctx_copy(ctx, g.data(), E.gram, sizeof(double) * 2 * nn, cudaMemcpyDeviceToHost));
  // upper block triangle (with the diagonal blocks) as computed, zeros below
  const int ld = 3 * m;
  for (int c = 0; c < ld; ++c)
    for (int r = 0; r < ld; ++r) {
      const bool upper = r / m <= c / m;
      const bool p_part = !has_p && (r >= 2 * m || c >= 2 * m);
      a[r + (size_t)c * ld] = (upper && !p_part) ? g[r + (size_t)c * ld] : 0.0;
      b[r + (size_t)c * ld] = (upper && !p_part) ? g[nn + r + (size_t)c * ld] : 0.0;
    }
  CK(ctx_copy(ctx, xtw, E.gxw, sizeof(double) * m * m, cudaMemcpyDeviceToHost));
  return DGDFT_OK;
}

template <class real>
dgdft_status lobpcg_update_t(dgdft_alb_ctx* ctx, int elem, int has_p, const double* blocks, const double* y,
                             double* out, int on_device) {
  Wave<real> w;
  dgdft_status s = with_step_wave<real>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  ElemDev<real>& E = w.h[0];
  const int m = E.m;
  const size_t n = (size_t)E.ng * m;
  const int order[6] = {BX, BW, BP, BHX, BHW, BHP};
  for (int q = 0; q < 6; ++q)
    if ((s = step_in<real>(ctx, E.blk[order[q]][0], blocks + q * n, n, on_device)) != DGDFT_OK) return s;
  for (int q = 0; q < 3 * m * m; ++q)
    if (!std::isfinite(y[q])) return ctx->fail(DGDFT_EINVAL, "lobpcg_update: non-finite coefficient");
  const int hp = has_p ? 1 : 0;
  CK(ctx_copy(ctx, E.state + ST_HAS_P, &hp, sizeof(int), cudaMemcpyHostToDevice));
  CK(ctx_copy(ctx, E.Y, y, sizeof(double) * 3 * m * m, cudaMemcpyHostToDevice));
  if (E.Yf) {
    std::vector<float> yf(3 * (size_t)m * m);
    for (size_t q = 0; q < yf.size(); ++q) yf[q] = (float)y[q];
    CK(ctx_copy(ctx, E.Yf, yf.data(), sizeof(float) * yf.size(), cudaMemcpyHostToDevice));
  }
  cudaStream_t st = ctx->stream;
  TsmmJob<real> t;
  t.nin = 3;
  t.in[0] = bref<real>(BX);
  t.in[1] = bref<real>(BW);
  t.in[2] = bref<real>(BP);
  t.yrow[0] = 0;
  t.yrow[1] = 1;
  t.yrow[2] = 2;
  t.needs_p[2] = 1;
  t.out = bref<real>(BX, 1);
  TsmmJob<real> u;
  u.nin = 2;
  u.in[0] = bref<real>(BW);
  u.in[1] = bref<real>(BP);
  u.yrow[0] = 1;
  u.yrow[1] = 2;
  u.needs_p[1] = 1;
  u.out = bref<real>(BP, 1);
  if (std::is_same<real, float>::value) {
    // as the FP32 stage: P' on the way to X'
    t.from2 = 1;
    t.out2 = bref<real>(BP, 1);
    w.update(t, st);
  } else {
    w.update(t, st);
    w.update(u, st);
  }
  u.in[0] = bref<real>(BHW);
  u.in[1] = bref<real>(BHP);
  u.out = bref<real>(BHP, 1);
  w.update(u, st);
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  int err = 0;
  CK(ctx_copy(ctx, &err, E.state + ST_ERROR, sizeof(int), cudaMemcpyDeviceToHost));
  if (err & ERR_TIMEOUT) return ctx->fail(DGDFT_ETIMEOUT, "lobpcg_update: a bounded device wait ran out");
  const int outs[3] = {BX, BP, BHP};
  for (int q = 0; q < 3; ++q)
    if ((s = step_out<real>(ctx, out + q * n, E.blk[outs[q]][1], n, on_device)) != DGDFT_OK) return s;
  return DGDFT_OK;
}

template <class real>
dgdft_status time_stage_t(dgdft_alb_ctx* ctx, Wave<real>& w, int stage, int reps, double* ms) {
  const int nel = (int)w.ids.size();
  std::vector<int> saved = w.h_state;
  for (int i = 0; i < nel; ++i) {
    std::vector<int> st(saved.begin() + (size_t)i * STATE_WORDS, saved.begin() + (size_t)(i + 1) * STATE_WORDS);
    st[ST_ACTIVE] = 1;
    st[ST_HAS_P] = 1;
    CK(ctx_copy(ctx, w.h[i].state, st.data(), sizeof(int) * STATE_WORDS, cudaMemcpyHostToDevice));
  }
  cudaStream_t st = ctx->stream;
  auto launch = [&]() {
    switch (stage) {
      case DGDFT_STAGE_XY_FWD: launch_h_pass<real>(w.batch, 0, bref<real>(BW), bref<real>(BHW), 0, st); break;
      case DGDFT_STAGE_Z_MULT: launch_h_pass<real>(w.batch, 1, bref<real>(BW), bref<real>(BHW), 0, st); break;
      case DGDFT_STAGE_XY_INV: launch_h_pass<real>(w.batch, 2, bref<real>(BW), bref<real>(BHW), 0, st); break;
      case DGDFT_STAGE_GRAM: w.gram_pencil(st); break;
      case DGDFT_STAGE_UPDATE: {
        TsmmJob<real> t;
        t.nin = 3;
        t.in[0] = bref<real>(BX);
        t.in[1] = bref<real>(BW);
        t.in[2] = bref<real>(BP);
        t.yrow[1] = 1;
        t.yrow[2] = 2;
        t.needs_p[2] = 1;
        t.out = bref<real>(BX, 1);
        w.update(t, st);
        break;
      }
      case DGDFT_STAGE_RR:
        launch_rr(w.d_rr_lob, nel, st, 3 * w.batch.s.max_m, w.batch.s.max_m, std::is_same<real, float>::value);
        break;
      default: launch_residual<real>(w.batch, w.rnchunk, st); break;
    }
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch();
  CK(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float el_ms = 0.0f;
  CK(cudaEventElapsedTime(&el_ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  *ms = (double)el_ms / reps;
  for (int i = 0; i < nel; ++i)
    CK(ctx_copy(ctx, w.h[i].state, &saved[(size_t)i * STATE_WORDS], sizeof(int) * STATE_WORDS,
                cudaMemcpyHostToDevice));
  return DGDFT_OK;
}

}  // namespace

extern "C" {

dgdft_status dgdft_alb_time_stage(dgdft_alb_ctx* ctx, int stage, int reps, double* ms_per_launch, int* n_elem,
                                  int* real_bytes) {
  if (!ctx || !ms_per_launch || stage < 0 || stage >= DGDFT_STAGE_COUNT || reps < 1) return DGDFT_EINVAL;
  if (!ctx->cache) return ctx->fail(DGDFT_ESTATE, "no resident wave: solve first (single-wave workloads)");
  CK(cudaSetDevice(ctx->device));
  WavePair* wp = static_cast<WavePair*>(ctx->cache);
  if (n_elem) *n_elem = (int)wp->w64->ids.size();
  if (wp->w32) {
    if (real_bytes) *real_bytes = 4;
    return time_stage_t<float>(ctx, *wp->w32, stage, reps, ms_per_launch);
  }
  if (real_bytes) *real_bytes = 8;
  return time_stage_t<double>(ctx, *wp->w64, stage, reps, ms_per_launch);
}

dgdft_status dgdft_alb_apply_h(dgdft_alb_ctx* ctx, int elem, int stage, int k, const double* x, double* hx,
                               int on_device) {
  if (!ctx || !x || !hx || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (k < 1 || k > ctx->el[elem].d.n_compute || (stage != 0 && stage != 1)) return DGDFT_EINVAL;
  return (ctx->cfg.precision == DGDFT_PREC_FP64 || stage == 1) ? apply_h_t<double>(ctx, elem, k, x, hx, on_device)
                                                               : apply_h_t<float>(ctx, elem, k, x, hx, on_device);
}

dgdft_status dgdft_alb_apply_teter(dgdft_alb_ctx* ctx, int elem, int k, const double* r, const double* t_kin,
                                   double* w, int on_device) {
  if (!ctx || !r || !t_kin || !w || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (k < 1 || k > ctx->el[elem].d.n_compute) return DGDFT_EINVAL;
  for (int i = 0; i < k; ++i)
    if (!(t_kin[i] > 0.0)) return DGDFT_EINVAL;
  return ctx->cfg.precision == DGDFT_PREC_FP64 ? teter_t<double>(ctx, elem, k, r, t_kin, w, on_device)
                                                : teter_t<float>(ctx, elem, k, r, t_kin, w, on_device);
}

dgdft_status dgdft_alb_project_cutoff(dgdft_alb_ctx* ctx, int elem, int k, const double* x, double* px,
                                      int on_device) {
  if (!ctx || !x || !px || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (k < 1 || k > ctx->el[elem].d.n_compute) return DGDFT_EINVAL;
  if (!(ctx->cfg.ecut > 0.0)) return ctx->fail(DGDFT_EINVAL, "project_cutoff: no planewave cutoff (ecut = 0)");
  return project_t(ctx, elem, k, x, px, on_device);
}

dgdft_status dgdft_alb_gram(dgdft_alb_ctx* ctx, int ng, int p, int q, const double* u, const double* v, double* c,
                            int on_device) {
  if (!ctx || !u || !v || !c || ng < 1 || p < 1 || q < 1) return DGDFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  return ctx->cfg.precision == DGDFT_PREC_FP64 ? gram_t<double>(ctx, ng, p, q, u, v, c, on_device)
                                                : gram_t<float>(ctx, ng, p, q, u, v, c, on_device);
}

dgdft_status dgdft_alb_lobpcg_gram(dgdft_alb_ctx* ctx, int elem, int stage, int has_p, const double* blocks,
                                   double* a, double* b, double* xtw, int on_device) {
  if (!ctx || !blocks || !a || !b || !xtw || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (stage != 0 && stage != 1) return DGDFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  return (ctx->cfg.precision == DGDFT_PREC_FP64 || stage == 1)
             ? lobpcg_gram_t<double>(ctx, elem, has_p, blocks, a, b, xtw, on_device)
             : lobpcg_gram_t<float>(ctx, elem, has_p, blocks, a, b, xtw, on_device);
}

dgdft_status dgdft_alb_lobpcg_update(dgdft_alb_ctx* ctx, int elem, int stage, int has_p, const double* blocks,
                                     const double* y, double* out, int on_device) {
  if (!ctx || !blocks || !y || !out || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  if (stage != 0 && stage != 1) return DGDFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  return (ctx->cfg.precision == DGDFT_PREC_FP64 || stage == 1)
             ? lobpcg_update_t<double>(ctx, elem, has_p, blocks, y, out, on_device)
             : lobpcg_update_t<float>(ctx, elem, has_p, blocks, y, out, on_device);
}

dgdft_status dgdft_alb_rayleigh_ritz(dgdft_alb_ctx* ctx, int stage, int n, int m, const double* a, const double* b,
                                     double* theta, double* y) {
  if (!ctx || !a || !b || !theta || !y || n < 1 || m < 1 || m > n) return DGDFT_EINVAL;
  if (stage != 0 && stage != 1) return DGDFT_EINVAL;
  const bool dfloat = stage == 0 && ctx->cfg.precision == DGDFT_PREC_MIXED;
  CK(cudaSetDevice(ctx->device));
  const size_t nn = (size_t)n * n;
  double *da = nullptr, *db = nullptr, *dy = nullptr, *dth = nullptr, *work = nullptr;
  RRTask* dt = nullptr;
  CK(cudaMalloc(&da, sizeof(double) * nn));
  CK(cudaMalloc(&db, sizeof(double) * nn));
  CK(cudaMalloc(&dy, sizeof(double) * (size_t)n * m));
  CK(cudaMalloc(&dth, sizeof(double) * m));
  CK(cudaMalloc(&work, sizeof(double) * rr_work_doubles(n, m)));
  CK(cudaMalloc(&dt, sizeof(RRTask)));
  RRTask t{};
  t.A = da;
  t.B = db;
  t.ld = n;
  t.mode = RR_FIXED;
  t.n_fixed = n;
  t.m = m;
  t.Y = dy;
  t.ldy = n;
  t.theta = dth;
  t.work = work;
  t.state = nullptr;
  t.cond_max = 1e30;
  dgdft_status s = DGDFT_OK;
  cudaError_t e = ctx_copy(ctx, da, a, sizeof(double) * nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ctx_copy(ctx, db, b, sizeof(double) * nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ctx_copy(ctx, dt, &t, sizeof(t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_rr(dt, 1, ctx->stream, n, m, dfloat);
    e = cudaStreamSynchronize(ctx->stream);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = ctx_copy(ctx, theta, dth, sizeof(double) * m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = ctx_copy(ctx, y, dy, sizeof(double) * (size_t)n * m, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) s = ctx->fail(DGDFT_ECUDA, "rayleigh_ritz: " + cuda_err_string(e));
  cudaFree(da);
  cudaFree(db);
  cudaFree(dy);
  cudaFree(dth);
  cudaFree(work);
  cudaFree(dt);
  if (s == DGDFT_OK && !std::isfinite(theta[0])) s = ctx->fail(DGDFT_EINVAL, "B is not positive definite");
  return s;
}

dgdft_status dgdft_alb_restrict_orthonormalise(dgdft_alb_ctx* ctx, int elem, int k, int J, const double* x,
                                               double* phi, int on_device) {
  if (!ctx || !x || !phi || elem < 0 || elem >= (int)ctx->el.size()) return DGDFT_EINVAL;
  ElemHost& eh = ctx->el[elem];
  if (k < 1 || k > eh.d.n_compute || J < 1 || J > k || J > eh.ne()) return DGDFT_EINVAL;
  Wave<double> w;
  dgdft_status s = with_step_wave<double>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  double* xs = w.h[0].blk[BW][0];
  if ((s = step_in<double>(ctx, xs, x, (size_t)eh.ng() * k, on_device)) != DGDFT_OK) return s;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * (size_t)eh.ne() * J));
  std::unique_ptr<void, decltype(&cudaFree)> guard(out, &cudaFree);
  if ((s = alb_orthonormalise(ctx, w, 0, xs, J, ctx->cfg.restrict_all ? k : J, out)) != DGDFT_OK) return s;
  CK(ctx_copy(ctx, phi, out, sizeof(double) * (size_t)eh.ne() * J,
                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return DGDFT_OK;
}

}  // extern "C"

// ------------------------------------------------ learned preconditioner

namespace {

dgdft_status ensure_net(dgdft_alb_ctx* ctx, uint64_t seed, bool reinit) {
  CK(cudaSetDevice(ctx->device));
  if (!ctx->net) ctx->net = new ConvNet();
  if (!ctx->net->ready || reinit) {
    std::string e = ctx->net->init(seed, ctx->stream);
    if (!e.empty()) return ctx->fail(DGDFT_ENOMEM, e);
  }
  return DGDFT_OK;
}

// A device view of caller data: the caller's pointer when on_device, else a
// temporary device copy (freed by the guard).
struct DevView {
  const void* ptr = nullptr;
  void* owned = nullptr;
  ~DevView() {
    if (owned) cudaFree(owned);
  }
};

dgdft_status dev_view(dgdft_alb_ctx* ctx, const void* src, size_t bytes, int on_device, DevView& v) {
  if (on_device) {
    v.ptr = src;
    return DGDFT_OK;
  }
  CK(cudaMalloc(&v.owned, bytes));
  CK(ctx_copy(ctx, v.owned, src, bytes, cudaMemcpyHostToDevice));
  v.ptr = v.owned;
  return DGDFT_OK;
}

}  // namespace

extern "C" {

dgdft_status dgdft_alb_precond_init(dgdft_alb_ctx* ctx, uint64_t seed) {
  if (!ctx) return DGDFT_EINVAL;
  return ensure_net(ctx, seed, true);
}

dgdft_status dgdft_alb_precond_set_params(dgdft_alb_ctx* ctx, const float* params) {
  if (!ctx || !params) return DGDFT_EINVAL;
  for (size_t i = 0; i < convnet_total_params(); ++i)
    if (!std::isfinite(params[i])) return ctx->fail(DGDFT_EINVAL, "non-finite network parameter");
  dgdft_status s = ensure_net(ctx, 0, false);
  if (s != DGDFT_OK) return s;
  std::string e = ctx->net->set_params(params, ctx->stream);
  return e.empty() ? DGDFT_OK : ctx->fail(DGDFT_ECUDA, e);
}

dgdft_status dgdft_alb_precond_get_params(dgdft_alb_ctx* ctx, float* params) {
  if (!ctx || !params) return DGDFT_EINVAL;
  if (!ctx->net || !ctx->net->ready) return ctx->fail(DGDFT_ESTATE, "no network");
  std::string e = ctx->net->get_params(params, ctx->stream);
  return e.empty() ? DGDFT_OK : ctx->fail(DGDFT_ECUDA, e);
}

dgdft_status dgdft_alb_precond_save(dgdft_alb_ctx* ctx, const char* path) {
  if (!ctx || !path) return DGDFT_EINVAL;
  if (!ctx->net || !ctx->net->ready) return ctx->fail(DGDFT_ESTATE, "no network");
  std::string e = ctx->net->save_file(path, ctx->stream);
  return e.empty() ? DGDFT_OK : ctx->fail(DGDFT_EINVAL, e);
}

dgdft_status dgdft_alb_precond_load(dgdft_alb_ctx* ctx, const char* path) {
  if (!ctx || !path) return DGDFT_EINVAL;
  dgdft_status s = ensure_net(ctx, 0, false);
  if (s != DGDFT_OK) return s;
  std::string e = ctx->net->load_file(path, ctx->stream);
  return e.empty() ? DGDFT_OK : ctx->fail(DGDFT_EINVAL, e);
}

dgdft_status dgdft_alb_precond_forward(dgdft_alb_ctx* ctx, int B, int nz, int ny, int nx, const float* in,
                                       float* out, int on_device) {
  if (!ctx || !in || !out || B < 1 || nz < 1 || ny < 1 || nx < 1) return DGDFT_EINVAL;
  if (!ctx->net || !ctx->net->ready) return ctx->fail(DGDFT_ESTATE, "no network");
  const size_t pts = (size_t)nz * ny * nx;
  DevView vin;
  dgdft_status s = dev_view(ctx, in, sizeof(float) * 2 * B * pts, on_device, vin);
  if (s != DGDFT_OK) return s;
  float *tmp = nullptr, *dout = nullptr;
  CK(cudaMalloc(&tmp, sizeof(float) * (2 * (size_t)B * 16 * pts + (size_t)B * pts)));
  std::unique_ptr<void, decltype(&cudaFree)> guard(tmp, &cudaFree);
  dout = tmp + 2 * (size_t)B * 16 * pts;
  ctx->net->forward((const float*)vin.ptr, dout, B, nz, ny, nx, nullptr, tmp, tmp + (size_t)B * 16 * pts,
                    ctx->stream);
  CK(cudaGetLastError());
  CK(ctx_copy(ctx, out, dout, sizeof(float) * B * pts, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return DGDFT_OK;
}

dgdft_status dgdft_alb_precond_loss_grad(dgdft_alb_ctx* ctx, int B, int nz, int ny, int nx, int lo, int hi,
                                         const float* in, const float* tgt, double* loss, float* grads,
                                         int on_device) {
  if (!ctx || !in || !tgt || !loss || !grads || B < 1 || nz < 1 || ny < 1 || nx < 1) return DGDFT_EINVAL;
  if (lo < 0 || hi <= lo || hi > nz || hi > ny || hi > nx) return DGDFT_EINVAL;
  if (!ctx->net || !ctx->net->ready) return ctx->fail(DGDFT_ESTATE, "no network");
  const size_t pts = (size_t)nz * ny * nx;
  DevView vin, vt;
  dgdft_status s = dev_view(ctx, in, sizeof(float) * 2 * B * pts, on_device, vin);
  if (s == DGDFT_OK) s = dev_view(ctx, tgt, sizeof(float) * B * pts, on_device, vt);
  if (s != DGDFT_OK) return s;
  std::string e = ctx->net->loss_and_grad((const float*)vin.ptr, (const float*)vt.ptr, B, nz, ny, nx, lo, hi, loss,
                                          ctx->stream);
  if (!e.empty()) return ctx->fail(DGDFT_ECUDA, e);
  size_t off = 0;
  for (int l = 0; l < kConvLayers; ++l) {
    const size_t n = conv_param_count(l);
    CK(ctx_copy(ctx, grads + off, ctx->net->grad[l], n * sizeof(float), cudaMemcpyDeviceToHost));
    off += n;
  }
  return DGDFT_OK;
}

dgdft_status dgdft_alb_precond_train(dgdft_alb_ctx* ctx, int nfields, int nz, int ny, int nx, const float* r,
                                     const float* v, const float* t, int crop, int batch, int steps, double lr,
                                     uint64_t seed, double* loss_first, double* loss_last) {
  if (!ctx || !r || !v || !t || nfields < 1 || crop < 9 || batch < 1 || steps < 1 || !(lr > 0.0))
    return DGDFT_EINVAL;
  dgdft_status s = ensure_net(ctx, seed, false);
  if (s != DGDFT_OK) return s;
  const size_t pts = (size_t)nz * ny * nx, cpts = (size_t)crop * crop * crop;
  float* buf = nullptr;
  CK(cudaMalloc(&buf, sizeof(float) * (3 * (size_t)batch * cpts + nfields) + sizeof(int) * 4 * batch));
  std::unique_ptr<void, decltype(&cudaFree)> guard(buf, &cudaFree);
  float* in = buf;
  float* tgt = in + 2 * (size_t)batch * cpts;
  float* rms = tgt + (size_t)batch * cpts;
  int* offs = reinterpret_cast<int*>(rms + nfields);
  field_rms(r, nfields, pts, rms, ctx->stream);
  std::mt19937_64 gen(seed ^ 0x5DEECE66DULL);
  std::vector<int> h_offs(4 * (size_t)batch);
  double first = 0.0, last = 0.0;
  const int avg = std::min(10, steps);
  for (int it = 0; it < steps; ++it) {
    for (int b = 0; b < batch; ++b) {
      h_offs[4 * b] = (int)(gen() % (uint64_t)nfields);
      h_offs[4 * b + 1] = (int)(gen() % (uint64_t)nz);
      h_offs[4 * b + 2] = (int)(gen() % (uint64_t)ny);
      h_offs[4 * b + 3] = (int)(gen() % (uint64_t)nx);
    }
    CK(cudaMemcpyAsync(offs, h_offs.data(), sizeof(int) * 4 * batch, cudaMemcpyHostToDevice, ctx->stream));
    gather_crops(r, v, t, rms, offs, batch, crop, nz, ny, nx, in, tgt, ctx->stream);
    double loss = 0.0;
    std::string e = ctx->net->loss_and_grad(in, tgt, batch, crop, crop, crop, 4, crop - 4, &loss, ctx->stream);
    if (!e.empty()) return ctx->fail(DGDFT_ECUDA, e);
    if (!std::isfinite(loss)) return ctx->fail(DGDFT_ENOTCONV, "training loss is not finite");
    ctx->net->adam((float)lr, ctx->stream);
    if (it < avg) first += loss / avg;
    if (it >= steps - avg) last += loss / avg;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  if (loss_first) *loss_first = first;
  if (loss_last) *loss_last = last;
  return DGDFT_OK;
}

dgdft_status dgdft_alb_precond_make_data(dgdft_alb_ctx* ctx, int elem, int nsnap, const int* snap_iters,
                                         float* r_out, float* t_out, double* sigma_out, int* cg_iters) {
  if (!ctx || !snap_iters || !r_out || !t_out || nsnap < 1 || elem < 0 || elem >= (int)ctx->el.size())
    return DGDFT_EINVAL;
  for (int q = 0; q < nsnap; ++q)
    if (snap_iters[q] < 1) return DGDFT_EINVAL;
  Wave<double> w;
  dgdft_status s = with_step_wave<double>(ctx, elem, w);
  if (s != DGDFT_OK) return s;
  ElemDev<double>& E = w.h[0];
  const int ng = E.ng, m = E.m;
  const size_t nb = (size_t)ng * m;
  cudaStream_t st = ctx->stream;
  double* small = nullptr;
  CK(cudaMalloc(&small, sizeof(double) * (64 * (size_t)m + 7 * (size_t)m)));
  std::unique_ptr<void, decltype(&cudaFree)> guard(small, &cudaFree);
  double* part = small;
  double* rr = part + 64 * m;
  double* rrn = rr + m;
  double* pap = rrn + m;
  double* alpha = pap + m;
  double* nalpha = alpha + m;
  double* beta = nalpha + m;
  double* negsig = beta + m;
  for (int q = 0; q < nsnap; ++q) {
    if ((s = w.load_inputs()) != DGDFT_OK) return s;
    if ((s = w.run(0.0, snap_iters[q], 0, nullptr)) != DGDFT_OK) return s;
    double theta0 = 0.0;
    CK(ctx_copy(ctx, &theta0, E.theta, sizeof(double), cudaMemcpyDeviceToHost));
    const double sigma = theta0 - 1.0;
    if (sigma_out) sigma_out[q] = sigma;
    double* R = E.blk[BW][0];
    launch_convert<double, float>(R, r_out + (size_t)q * nb, nb, st);
    // CG on (H - sigma I) t = r for all m columns at once
    if ((s = w.reset_states(0.0)) != DGDFT_OK) return s;
    double* T = E.blk[BP][1];
    double* RC = E.blk[BHW][0];
    double* P = E.blk[BHP][1];
    double* AP = E.blk[BP][0];
    CK(cudaMemsetAsync(T, 0, sizeof(double) * nb, st));
    CK(cudaMemcpyAsync(RC, R, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(P, R, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
    std::vector<double> hs(m, -sigma);
    CK(cudaMemcpyAsync(negsig, hs.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    col_dot(RC, RC, ng, m, part, rr, st);
    std::vector<double> b2(m), cur(m);
    CK(ctx_copy(ctx, b2.data(), rr, sizeof(double) * m, cudaMemcpyDeviceToHost));
    int it = 0;
    for (; it < 1000; ++it) {
      launch_apply_h<double>(w.batch, bptr<double>(P), bptr<double>(AP), m, st);
      col_axpby(negsig, P, nullptr, AP, ng, m, st);
      col_dot(P, AP, ng, m, part, pap, st);
      cg_alpha(rr, pap, alpha, nalpha, m, st);
      col_axpby(alpha, P, nullptr, T, ng, m, st);
      col_axpby(nalpha, AP, nullptr, RC, ng, m, st);
      col_dot(RC, RC, ng, m, part, rrn, st);
      cg_beta(rr, rrn, beta, m, st);
      col_axpby(nullptr, RC, beta, P, ng, m, st);
      if (it % 10 == 9) {
        CK(ctx_copy(ctx, cur.data(), rr, sizeof(double) * m, cudaMemcpyDeviceToHost));
        double worst = 0.0;
        for (int j = 0; j < m; ++j) worst = std::max(worst, std::sqrt(cur[j] / std::max(b2[j], 1e-300)));
        if (worst <= 1e-10) break;
      }
    }
    CK(cudaGetLastError());
    if (cg_iters) cg_iters[q] = it + 1;
    launch_convert<double, float>(T, t_out + (size_t)q * nb, nb, st);
    CK(cudaStreamSynchronize(st));
  }
  return DGDFT_OK;
}

}  // extern "C"
