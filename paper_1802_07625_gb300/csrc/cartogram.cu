// C-ABI of the cartogram library: context, validation, device memory, the CUDA graph
// of one integration, and the outer iteration. Declarations and their contracts are
// in include/cartogram.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cartogram.h"
#include "ff.cuh"
#include "kernels.h"

using cg::DevState;
using cg::IterInfo;
using cg::StepParams;
using cg::V2;

// Device workspace of the iteration gradient (FP64), allocated on first use.
struct AdjWork {
  int C = 0;                     // steps between checkpoints
  double2* lam = nullptr;        // adjoint of the displacements [N]
  double* L[2] = {nullptr, nullptr};  // field adjoints of two time levels [N][2]
  double *a_rho = nullptr, *a_gx = nullptr, *a_gy = nullptr;  // node adjoints [N]
  double *Crho = nullptr, *Cx = nullptr, *Cy = nullptr;       // their DCT-II [N]
  double *lam_spec = nullptr, *specp = nullptr, *R = nullptr, *dens = nullptr;  // [N]
  double2* AB = nullptr;         // inverse-pass intermediate [N]
  // the three transposed transforms of a level run side by side (each fills a fraction of
  // the GPU): the second and third on their own streams with their own intermediates
  double* R2[2] = {nullptr, nullptr};  // [N] each
  double2* AB2[2] = {nullptr, nullptr};  // inverse-pass intermediates of the side streams [N] each
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  double2* Dk = nullptr;         // final displacements of the iteration being reversed [N]
  double2* flux = nullptr;       // inverse-pass side output [N]
  std::vector<double2*> v;       // fields of a segment's levels [C + 1][N]
  std::vector<double*> rho;      // densities of a segment's levels [C + 1][N]
  std::vector<double2*> D;       // displacements of a segment's levels [C + 1][N]
  std::vector<double2*> ckpt;    // checkpointed displacements
  double* sched = nullptr;       // recorded (t, h), [max_steps][2]
  double* vals = nullptr;        // target values of the call [R]
  double* dLdA = nullptr;        // [R]
  double* gw = nullptr;          // d L / d w [R]
  double* dsig = nullptr;        // [1]
  double2* xy1 = nullptr;        // mapped vertices [n_vert]
  double2* gv = nullptr;         // their adjoints [n_vert]
  double2* gv2 = nullptr;        // [n_vert]
  std::vector<double2*> X;       // vertices entering each iteration, [K + 1][n_vert]
  std::vector<double*> spec;     // each iteration's spectrum, [K][N]
  long long n_vert = 0;
  int n_regions = 0;
};

struct cg_ctx {
  int Lx = 0, Ly = 0, log2Lx = 0, log2Ly = 0;
  double blur = 0.0;
  cg_options opt{};
  bool mixed = false;
  bool ff = false;  // CG_PRECISION_MIXED_FF: pass 2 in float-float arithmetic
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;

  // transform tables: inverse roots and quarter-wave factors in the working type,
  // forward (FP64) roots, quarter-wave factors and blur factors
  void *Wx = nullptr, *Wy = nullptr, *Ex = nullptr, *Ey = nullptr;
  void *Wyff = nullptr, *Eyff = nullptr;  // float-float pass-2 tables (CG_PRECISION_MIXED_FF)
  // float-float forward roots and quarter-wave factors of both axes (the mixed precisions'
  // forward transform)
  void *Wfxff = nullptr, *Efxff = nullptr, *Wfyff = nullptr, *Efyff = nullptr;
  int ff_cols_max = 0;                    // largest block of the float-float pass 2
  double2 *Wfx = nullptr, *Wfy = nullptr, *Efx = nullptr, *Efy = nullptr;
  double *bx = nullptr, *by = nullptr;  // blur factors for width blur_tab_sigma
  double blur_tab_sigma = -1.0;           // -1: the tables hold no known width

  // fields
  double* acc = nullptr;     // rasterised rho/rho_bar - 1 (FP64)
  double* R = nullptr;       // forward transform along x
  double* spec64 = nullptr;  // blurred cosine spectrum (FP64), (0,0) removed
  void* specT = nullptr;     // spectrum in the working type (aliases spec64 in FP64)
  void* AB = nullptr;        // pass-1 output
  void* vbuf[2] = {nullptr, nullptr};
  void* dbuf[2] = {nullptr, nullptr};
  void* ubuf[2] = {nullptr, nullptr};  // cached predictor velocities, by parity like dbuf
  void* dres = nullptr;      // displacements of the last integration
  void* rho_tmp = nullptr;   // density output of the field entry point
  void* phi = nullptr;       // linear flow: Phi~ = rho~ / (pi^2 k^2) in the working type
  void* flux = nullptr;      // linear flow: J = -grad Phi at the cell centres
  void* rho0 = nullptr;      // linear flow: initial density at the cell centres
  DevState* st = nullptr;
  unsigned long long* deadline = nullptr;  // device-clock deadline of the call in flight (0: none)
  IterInfo* info = nullptr;
  IterInfo* info_h = nullptr;  // pinned
  bool have_spectrum = false;

  // map
  bool have_regions = false;
  int R_n = 0;
  long long n_rings = 0, n_vert = 0;
  double* values = nullptr;
  long long* ring_off = nullptr;
  int* reg_off = nullptr;
  int* reg_rings = nullptr;
  int* chunk_ring = nullptr;      // area sums: the ring of every vertex chunk
  int* ring_chunk_off = nullptr;  // ring k's chunks are [ring_chunk_off[k], ring_chunk_off[k+1])
  double* chunk_sum = nullptr;    // one shoelace partial sum per chunk
  long long n_chunks = 0;
  int* next = nullptr;
  int* vreg = nullptr;
  double2* xy = nullptr;
  double2* xy0 = nullptr;  // vertices as given to set_regions
  double* area_sums = nullptr;  // (sum A, sum V) of the last area computation
  std::vector<long long> map_off;  // host copies of the map's ring offsets and ring regions:
  std::vector<int> map_reg;        // a new map with the same rings reuses every buffer
  double* area = nullptr;
  double* err_d = nullptr;
  double* w = nullptr;
  std::vector<void*> hist;
  int hist_len = 0;
  double2* pts = nullptr;
  long long pts_cap = 0;
  double* diag = nullptr;  // distortion scratch: per-block sums, maxima, results
  int* prev = nullptr;     // ring predecessor of every vertex
  double* sched_rec = nullptr;      // while recording: (t, h) of the accepted steps (device)
  std::vector<std::vector<double>> scheds;  // the last recorded schedules, per iteration [n][2]
  AdjWork* adj = nullptr;           // workspace of the iteration gradient

  // persistent integration kernel
  cg::GridBarrier* gb = nullptr;
  cg::StepAcc* acc2 = nullptr;  // two reduction slots
  int persist_grid = 0;         // 0: not available
  size_t persist_smem = 0;
  int persist_rows = 0, persist_cols = 0;

  // launch shapes of the step kernels
  cg::Tune tune;
  bool tuned = false;
  double tune_ms[3] = {0, 0, 0};

  // graph of one integration
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // the outer iteration on the device: one graph launch runs iterations until the areas
  // converge (or the budget, a failure, or the free history slots end it)
  cg::OuterState* outer = nullptr;    // device
  cg::OuterState* outer_h = nullptr;  // pinned
  double* sigma_d = nullptr;          // blur width per iteration of a call
  double* sigma_h = nullptr;          // pinned
  int sigma_cap = 0;
  void** hist_d = nullptr;            // device copy of the history slot pointers
  int hist_d_cap = 0;
  int hist_d_count = 0;               // pointers in hist_d
  cudaGraph_t ograph = nullptr;
  cudaGraphExec_t oexec = nullptr;
  unsigned long long gen = 1;         // changes whenever captured graphs of this context go stale
};

// Independent contexts whose outer iterations run as parallel branches of one graph.
struct cg_batch {
  std::vector<cg_ctx*> ctx;
  std::vector<unsigned long long> gen;  // each context's generation when the graph was built
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {

int fail(cg_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

#define CG_CUDA(ctx, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
  } while (0)

bool pow2_in_range(int n) { return n >= 8 && n <= 1024 && (n & (n - 1)) == 0; }
int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Start of a call: the deadline is the device clock now plus the time limit (0: none).
void stamp_deadline(cg_ctx* c, bool limited = true) {
  const double ns = limited ? c->opt.time_limit * 1e9 : 0.0;
  cg::launch_deadline(c->deadline, ns > 0.0 ? (unsigned long long)ns + 1ull : 0ull, c->stream);
}

// Bit pattern of the largest x >= 0 with sqrt(x) <= atol (double arithmetic; sqrt is
// correctly rounded on host and device alike): the step controller's accept test on the
// squared error.
unsigned long long err2_accept_bits(double atol) {
  double x = atol * atol;
  for (int k = 0; k < 64 && x < HUGE_VAL && std::sqrt(std::nextafter(x, HUGE_VAL)) <= atol; ++k)
    x = std::nextafter(x, HUGE_VAL);
  for (int k = 0; k < 64 && x > 0.0 && std::sqrt(x) > atol; ++k) x = std::nextafter(x, 0.0);
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
}

cg::AreaChunks area_chunks(const cg_ctx* c) {
  cg::AreaChunks ch;
  ch.chunk_ring = c->chunk_ring;
  ch.ring_chunk_off = c->ring_chunk_off;
  ch.n_chunks = c->n_chunks;
  ch.chunk_sum = c->chunk_sum;
  return ch;
}

StepParams step_params(const cg_ctx* c) {
  StepParams sp;
  sp.err2_accept_bits = err2_accept_bits(c->opt.atol);
  sp.dt0 = c->opt.dt0;
  sp.atol = c->opt.atol;
  sp.grow = c->opt.grow;
  sp.shrink = c->opt.shrink;
  sp.cfl = c->opt.cfl;
  sp.rho_tol = c->opt.rho_tol;
  sp.h_min = 0.0;
  sp.max_steps = c->opt.max_steps;
  sp.sched = c->sched_rec;
  sp.deadline = c->deadline;
  return sp;
}

template <typename T>
int upload_tables(cg_ctx* c, int N, void** Wd, void** Ed, double2** Wfd, double2** Efd) {
  // inter-step twiddles of the four-step FFT in [k2][n1] order, TW[k2*N1 + n1] =
  // exp(+-2 pi i n1 k2 / N), and quarter-wave factors E[m] = exp(i pi m/(2N)); the
  // angles are reduced exactly on the integers before the library cos/sin
  const int log2N = ilog2(N);
  const int N1 = 1 << ((log2N + 1) / 2), N2 = N / N1;
  std::vector<V2<T>> W(N), E(N);
  std::vector<double2> Wf(N), Ef(N);
  for (int k2 = 0; k2 < N2; ++k2)
    for (int n1 = 0; n1 < N1; ++n1) {
      const int p = (n1 * k2) % N;
      const double a = 2.0 * cg::kPi * (double)p / N;
      const double cw = std::cos(a), sw = std::sin(a);
      W[k2 * N1 + n1].x = (T)cw;
      W[k2 * N1 + n1].y = (T)sw;
      Wf[k2 * N1 + n1] = make_double2(cw, -sw);
    }
  for (int p = 0; p < N; ++p) {
    const double b = cg::kPi * (double)p / (2.0 * N);
    const double ce = std::cos(b), se = std::sin(b);
    E[p].x = (T)ce;
    E[p].y = (T)se;
    Ef[p] = make_double2(ce, se);
  }
  CG_CUDA(c, cudaMalloc(Wd, sizeof(V2<T>) * N));
  CG_CUDA(c, cudaMalloc(Ed, sizeof(V2<T>) * N));
  CG_CUDA(c, cudaMalloc((void**)Wfd, sizeof(double2) * N));
  CG_CUDA(c, cudaMalloc((void**)Efd, sizeof(double2) * N));
  CG_CUDA(c, cudaMemcpy(*Wd, W.data(), sizeof(V2<T>) * N, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(*Ed, E.data(), sizeof(V2<T>) * N, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(*Wfd, Wf.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(*Efd, Ef.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
  return CG_OK;
}

// The pass-2 tables of the compensated mixed precision: the same inter-step twiddles and
// quarter-wave factors as upload_tables, each as the float-float pair nearest the FP64 value.
int upload_tables_ff(cg_ctx* c, int N, void** Wd, void** Ed) {
  const int log2N = ilog2(N);
  const int N1 = 1 << ((log2N + 1) / 2), N2 = N / N1;
  std::vector<cg::ff2> W(N), E(N);
  for (int k2 = 0; k2 < N2; ++k2)
    for (int n1 = 0; n1 < N1; ++n1) {
      const double a = 2.0 * cg::kPi * (double)((n1 * k2) % N) / N;
      W[k2 * N1 + n1].x = cg::ff(std::cos(a));
      W[k2 * N1 + n1].y = cg::ff(std::sin(a));
    }
  for (int p = 0; p < N; ++p) {
    const double b = cg::kPi * (double)p / (2.0 * N);
    E[p].x = cg::ff(std::cos(b));
    E[p].y = cg::ff(std::sin(b));
  }
  CG_CUDA(c, cudaMalloc(Wd, sizeof(cg::ff2) * N));
  CG_CUDA(c, cudaMalloc(Ed, sizeof(cg::ff2) * N));
  CG_CUDA(c, cudaMemcpy(*Wd, W.data(), sizeof(cg::ff2) * N, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(*Ed, E.data(), sizeof(cg::ff2) * N, cudaMemcpyHostToDevice));
  return CG_OK;
}

// The forward-transform tables of the mixed precisions: the forward roots exp(-2 pi i n1 k2 /
// N) and the quarter-wave factors exp(i pi m / (2N)), each as the float-float pair nearest the
// FP64 value.
int upload_fwd_tables_ff(cg_ctx* c, int N, void** Wd, void** Ed) {
  const int log2N = ilog2(N);
  const int N1 = 1 << ((log2N + 1) / 2), N2 = N / N1;
  std::vector<cg::ff2> W(N), E(N);
  for (int k2 = 0; k2 < N2; ++k2)
    for (int n1 = 0; n1 < N1; ++n1) {
      const double a = 2.0 * cg::kPi * (double)((n1 * k2) % N) / N;
      W[k2 * N1 + n1].x = cg::ff(std::cos(a));
      W[k2 * N1 + n1].y = cg::ff(-std::sin(a));
    }
  for (int p = 0; p < N; ++p) {
    const double b = cg::kPi * (double)p / (2.0 * N);
    E[p].x = cg::ff(std::cos(b));
    E[p].y = cg::ff(std::sin(b));
  }
  CG_CUDA(c, cudaMalloc(Wd, sizeof(cg::ff2) * N));
  CG_CUDA(c, cudaMalloc(Ed, sizeof(cg::ff2) * N));
  CG_CUDA(c, cudaMemcpy(*Wd, W.data(), sizeof(cg::ff2) * N, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(*Ed, E.data(), sizeof(cg::ff2) * N, cudaMemcpyHostToDevice));
  return CG_OK;
}

// Separable blur factors exp(-(pi m / L)^2 sigma^2 / 2) of both axes, computed on the
// device by the same kernel the device-side outer iteration uses.
int set_blur_tables(cg_ctx* c, double sigma) {
  cg::launch_blur_tables(nullptr, sigma, c->bx, c->by, c->Lx, c->Ly, c->stream);
  CG_CUDA(c, cudaGetLastError());
  c->blur_tab_sigma = sigma;
  return CG_OK;
}

// The forward transform of the rasterised density c->acc into the spectrum (FP64, and its FP32
// copy for the mixed precisions, whose forward transform runs in float-float arithmetic).
template <typename T>
void launch_forward(cg_ctx* c, const double* bx, const double* by, cudaStream_t s) {
  if constexpr (sizeof(T) == 4)
    cg::launch_fwd_ff(c->log2Lx, c->log2Ly, c->acc, c->R, c->spec64, (float*)c->specT, c->Wfxff, c->Efxff,
                      c->Wfyff, c->Efyff, bx, by, s);
  else
    cg::launch_fwd<T>(c->log2Lx, c->log2Ly, c->acc, c->R, c->spec64, nullptr, c->Wfx, c->Efx, c->Wfy, c->Efy,
                      bx, by, s);
}

template <typename T>
int alloc_fields(cg_ctx* c) {
  const size_t N = (size_t)c->Lx * c->Ly;
  int r = upload_tables<T>(c, c->Lx, &c->Wx, &c->Ex, &c->Wfx, &c->Efx);
  if (r) return r;
  r = upload_tables<T>(c, c->Ly, &c->Wy, &c->Ey, &c->Wfy, &c->Efy);
  if (r) return r;
  if (c->ff) {
    if ((r = upload_tables_ff(c, c->Ly, &c->Wyff, &c->Eyff))) return r;
    CG_CUDA(c, cg::prepare_spectral_ff(c->log2Ly, c->Lx, &c->ff_cols_max));
  }
  if constexpr (sizeof(T) == 4) {
    if ((r = upload_fwd_tables_ff(c, c->Lx, &c->Wfxff, &c->Efxff))) return r;
    if ((r = upload_fwd_tables_ff(c, c->Ly, &c->Wfyff, &c->Efyff))) return r;
    CG_CUDA(c, cg::prepare_forward_ff(c->log2Lx, c->log2Ly));
  }
  CG_CUDA(c, cudaMalloc((void**)&c->bx, sizeof(double) * c->Lx));
  CG_CUDA(c, cudaMalloc((void**)&c->by, sizeof(double) * c->Ly));
  CG_CUDA(c, cudaMalloc((void**)&c->outer, sizeof(cg::OuterState)));
  CG_CUDA(c, cudaMallocHost((void**)&c->outer_h, sizeof(cg::OuterState)));
  if (c->blur > 0.0 && (r = set_blur_tables(c, c->blur))) return r;
  CG_CUDA(c, cudaMalloc((void**)&c->acc, sizeof(double) * N));
  CG_CUDA(c, cudaMalloc((void**)&c->R, sizeof(double) * N));
  CG_CUDA(c, cudaMalloc((void**)&c->spec64, sizeof(double) * N));
  if (sizeof(T) == 4) {
    CG_CUDA(c, cudaMalloc(&c->specT, sizeof(T) * N));
  } else {
    c->specT = c->spec64;
  }
  CG_CUDA(c, cudaMalloc(&c->AB, sizeof(V2<T>) * N));
  for (int k = 0; k < 2; ++k) {
    CG_CUDA(c, cudaMalloc(&c->vbuf[k], sizeof(V2<T>) * N));
    CG_CUDA(c, cudaMalloc(&c->dbuf[k], sizeof(V2<T>) * N));
    CG_CUDA(c, cudaMalloc(&c->ubuf[k], sizeof(V2<T>) * N));
  }
  CG_CUDA(c, cudaMalloc(&c->dres, sizeof(V2<T>) * N));
  CG_CUDA(c, cudaMemset(c->dres, 0, sizeof(V2<T>) * N));
  CG_CUDA(c, cudaMalloc(&c->rho_tmp, sizeof(T) * N));
  if (c->opt.flow == CG_FLOW_LINEAR) {
    CG_CUDA(c, cudaMalloc(&c->phi, sizeof(T) * N));
    CG_CUDA(c, cudaMalloc(&c->flux, sizeof(V2<T>) * N));
    CG_CUDA(c, cudaMalloc(&c->rho0, sizeof(T) * N));
  }
  CG_CUDA(c, cudaMalloc((void**)&c->st, sizeof(DevState)));
  CG_CUDA(c, cudaMemset(c->st, 0, sizeof(DevState)));
  CG_CUDA(c, cudaMalloc((void**)&c->deadline, sizeof(unsigned long long)));
  CG_CUDA(c, cudaMemset(c->deadline, 0, sizeof(unsigned long long)));
  CG_CUDA(c, cudaMalloc((void**)&c->info, sizeof(IterInfo)));
  CG_CUDA(c, cudaMallocHost((void**)&c->info_h, sizeof(IterInfo)));
  CG_CUDA(c, cudaMemset(c->spec64, 0, sizeof(double) * N));
  if (sizeof(T) == 4) CG_CUDA(c, cudaMemset(c->specT, 0, sizeof(T) * N));
  CG_CUDA(c, cg::prepare_spectral<T>(c->log2Lx, c->log2Ly));
  CG_CUDA(c, cg::prepare_forward(c->log2Lx, c->log2Ly));
  CG_CUDA(c, cudaMalloc((void**)&c->gb, sizeof(cg::GridBarrier)));
  CG_CUDA(c, cudaMalloc((void**)&c->acc2, 2 * sizeof(cg::StepAcc)));
  // the persistent kernel: one resident grid sized to the larger of the two passes
  {
    const int S = cg::default_rows(c->log2Lx, c->Ly), Wc = cg::default_cols(c->Lx, sizeof(T));
    const size_t smem = std::max(cg::inv_rows_cfg(c->log2Lx, c->Ly, sizeof(T), S).smem,
                                 cg::inv_cols_cfg(c->log2Ly, c->Lx, sizeof(T), Wc).smem);
    int bps = 0, coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    // (the persistent kernel runs the working type's pass 2 only: not for float-float)
    if (!c->ff && coop && smem <= 227 * 1024 && cg::prepare_integrate<T>(smem, &bps) == cudaSuccess && bps > 0) {
      const int items = std::max(c->Ly / S, c->Lx / Wc);
      c->persist_grid = std::min(bps * cg::sm_count(), std::max(items, cg::sm_count()));
      c->persist_smem = smem;
      c->persist_rows = S;
      c->persist_cols = Wc;
    }
    cudaGetLastError();
  }
  return CG_OK;
}

// ---- the kernels of one integration ------------------------------------------

// Pass 2 of the inverse transform with this context's arithmetic (float-float for the
// compensated mixed precision, the working type otherwise).
template <typename T>
void launch_cols(cg_ctx* c, int Wc, const V2<T>* AB, V2<T>* v0, V2<T>* v1, T* rho_out, int mode, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (c->ff) {
      cg::launch_inv_cols_ff(c->log2Ly, c->Lx, Wc, (const float2*)AB, (float2*)v0, (float2*)v1, (float*)rho_out,
                             c->Wyff, c->Eyff, c->st, mode, s);
      return;
    }
  }
  cg::launch_inv_cols<T>(c->log2Ly, c->Lx, Wc, AB, v0, v1, rho_out, (const V2<T>*)c->Wy, (const V2<T>*)c->Ey, c->st,
                         mode, s);
}

template <typename T>
void enqueue_field(cg_ctx* c, int mode, double tau, V2<T>* out0, V2<T>* out1, T* rho_out,
                   cudaStream_t s, cudaGraphConditionalHandle h = 0, int use_cond = 0) {
  cg::launch_inv_rows<T>(c->log2Lx, c->Ly, c->tune.rows, (const T*)c->specT, (V2<T>*)c->AB,
                         (const V2<T>*)c->Wx, (const V2<T>*)c->Ex, c->st, mode, tau, h, use_cond,
                         (unsigned int)c->opt.max_steps + 8u, s);
  launch_cols<T>(c, c->tune.cols, (const V2<T>*)c->AB, out0, out1, rho_out, mode, s);
}

template <typename T>
void enqueue_init(cg_ctx* c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  const StepParams sp = step_params(c);
  cg::launch_init_state(c->st, sp, s);
  cudaMemsetAsync(c->dbuf[0], 0, sizeof(V2<T>) * (size_t)c->Lx * c->Ly, s);
  enqueue_field<T>(c, cg::kModeInit, 0.0, (V2<T>*)c->vbuf[0], (V2<T>*)c->vbuf[1], nullptr, s);
  cg::launch_gather_u<T>((const V2<T>*)c->vbuf[0], (const V2<T>*)c->dbuf[0], (V2<T>*)c->ubuf[0], c->Lx, c->Ly, s);
  cg::launch_init_finish(c->st, sp, h, use_cond, s);
}

// Attempt k of a run of attempts that starts at an even attempt (its parity selects the
// state slot of the step loop).
template <typename T>
void enqueue_body(cg_ctx* c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s, int k) {
  const StepParams sp = step_params(c);
  const int mode = (k & 1) ? cg::kModeStepOdd : cg::kModeStep;
  enqueue_field<T>(c, mode, 0.0, (V2<T>*)c->vbuf[0], (V2<T>*)c->vbuf[1], nullptr, s, h, use_cond);
  cg::launch_heun<T>(c->st, sp, (const V2<T>*)c->vbuf[0], (const V2<T>*)c->vbuf[1],
                     (V2<T>*)c->dbuf[0], (V2<T>*)c->dbuf[1], (V2<T>*)c->ubuf[0], (V2<T>*)c->ubuf[1],
                     c->Lx, c->Ly, mode, 0.0, h, use_cond, c->tune.heun_bps, s);
}

// Linear flow, once per integration: Phi~, the flux J = -grad Phi and rho0 at the cell
// centres (transform passes at tau = 0), the speed at t = 0 and the first step.
template <typename T>
void enqueue_init_linear(cg_ctx* c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  const StepParams sp = step_params(c);
  cg::launch_init_state(c->st, sp, s);
  cudaMemsetAsync(c->dbuf[0], 0, sizeof(V2<T>) * (size_t)c->Lx * c->Ly, s);
  cg::launch_phi_spectrum<T>(c->spec64, (T*)c->phi, c->Lx, c->Ly, s);
  cg::launch_inv_rows<T>(c->log2Lx, c->Ly, c->tune.rows, (const T*)c->phi, (V2<T>*)c->AB,
                         (const V2<T>*)c->Wx, (const V2<T>*)c->Ex, c->st, cg::kModeFlux, 0.0, 0, 0, 0u, s);
  launch_cols<T>(c, c->tune.cols, (const V2<T>*)c->AB, (V2<T>*)c->flux, nullptr, nullptr, cg::kModeFlux, s);
  cg::launch_inv_rows<T>(c->log2Lx, c->Ly, c->tune.rows, (const T*)c->specT, (V2<T>*)c->AB,
                         (const V2<T>*)c->Wx, (const V2<T>*)c->Ex, c->st, cg::kModeFixed, 0.0, 0, 0, 0u, s);
  launch_cols<T>(c, c->tune.cols, (const V2<T>*)c->AB, (V2<T>*)c->vbuf[0], nullptr, (T*)c->rho0, cg::kModeFixed,
                 s);
  cudaMemsetAsync(&c->st->vmax2_bits, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(&c->st->dev_bits, 0, sizeof(unsigned long long), s);
  cg::launch_linear_init<T>(c->st, sp, (const V2<T>*)c->flux, (const T*)c->rho0, (V2<T>*)c->vbuf[0],
                            c->Lx * c->Ly, h, use_cond, s);
  cg::launch_gather_u<T>((const V2<T>*)c->vbuf[0], (const V2<T>*)c->dbuf[0], (V2<T>*)c->ubuf[0], c->Lx, c->Ly, s);
}

template <typename T>
void enqueue_body_linear(cg_ctx* c, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  cg::launch_linear_step<T>(c->st, step_params(c), (const V2<T>*)c->flux, (const T*)c->rho0,
                            (V2<T>*)c->vbuf[0], (V2<T>*)c->vbuf[1], (V2<T>*)c->dbuf[0], (V2<T>*)c->dbuf[1],
                            (V2<T>*)c->ubuf[0], (V2<T>*)c->ubuf[1], c->Lx, c->Ly, h, use_cond, (unsigned int)c->opt.max_steps + 8u, c->tune.heun_bps, s);
}

template <typename T>
void enqueue_finish(cg_ctx* c, cudaStream_t s) {
  cg::launch_snapshot<T>(c->st, (const V2<T>*)c->dbuf[0], (const V2<T>*)c->dbuf[1], (V2<T>*)c->dres,
                         c->Lx * c->Ly, s);
  cg::launch_collect(c->st, c->info, s);
}

void drop_outer_graph(cg_ctx* c);

// Time the candidate launch shapes of the three step kernels with CUDA events on the
// context's stream (fields of the current spectrum at fixed times, the displacements of
// the last integration) and keep the fastest of each.
template <typename T>
int do_autotune(cg_ctx* c, int reps) {
  cudaStream_t s = c->stream;
  const size_t esz = sizeof(T);
  cudaEvent_t a, b;
  CG_CUDA(c, cudaEventCreate(&a));
  CG_CUDA(c, cudaEventCreate(&b));
  CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  CG_CUDA(c, cudaMemcpyAsync(c->dbuf[0], c->dres, sizeof(V2<T>) * (size_t)c->Lx * c->Ly,
                             cudaMemcpyDeviceToDevice, s));
  const double t = 1.0, h = 0.5;
  enqueue_field<T>(c, cg::kModeFixed, t, (V2<T>*)c->vbuf[0], nullptr, nullptr, s);
  enqueue_field<T>(c, cg::kModeFixed, t + h, (V2<T>*)c->vbuf[1], nullptr, nullptr, s);
  auto timeit = [&](auto&& launch, double* ms) -> int {
    launch();
    *ms = 1e30;
    for (int round = 0; round < 3; ++round) {
      CG_CUDA(c, cudaEventRecord(a, s));
      for (int r = 0; r < reps; ++r) launch();
      CG_CUDA(c, cudaEventRecord(b, s));
      CG_CUDA(c, cudaEventSynchronize(b));
      float f = 0.f;
      CG_CUDA(c, cudaEventElapsedTime(&f, a, b));
      *ms = std::min(*ms, (double)f / reps);
    }
    return CG_OK;
  };
  cg::Tune best = c->tune;
  double best_ms[3] = {1e30, 1e30, 1e30};
  int r;
  int rows_max = 0, cols_max = 0;
  CG_CUDA(c, cg::spectral_max_threads<T>(c->log2Lx, c->log2Ly, &rows_max, &cols_max));
  for (int S = 1; S <= 16 && S <= c->Ly; S *= 2) {
    const cg::LaunchCfg k = cg::inv_rows_cfg(c->log2Lx, c->Ly, esz, S);
    if (k.smem > 227 * 1024 || k.threads > rows_max) continue;
    double ms;
    if ((r = timeit([&] {
           cg::launch_inv_rows<T>(c->log2Lx, c->Ly, S, (const T*)c->specT, (V2<T>*)c->AB,
                                  (const V2<T>*)c->Wx, (const V2<T>*)c->Ex, c->st, cg::kModeFixed,
                                  t + h, 0, 0, 0u, s);
         }, &ms)))
      return r;
    if (ms < best_ms[0]) { best_ms[0] = ms; best.rows = S; }
  }
  for (int W = 2; W <= 16 && W <= c->Lx; W *= 2) {
    const cg::LaunchCfg k = c->ff ? cg::inv_cols_ff_cfg(c->log2Ly, c->Lx, W) : cg::inv_cols_cfg(c->log2Ly, c->Lx, esz, W);
    if (k.smem > 227 * 1024 || k.threads > (c->ff ? c->ff_cols_max : cols_max)) continue;
    double ms;
    if ((r = timeit([&] {
           launch_cols<T>(c, W, (const V2<T>*)c->AB, (V2<T>*)c->vbuf[1], nullptr, nullptr, cg::kModeFixed, s);
         }, &ms)))
      return r;
    if (ms < best_ms[1]) { best_ms[1] = ms; best.cols = W; }
  }
  const StepParams sp = step_params(c);
  // resident blocks per SM of the step kernel: its 256-thread blocks fit five to an SM at
  // 48 registers, so the counts around that are tried too
  cg::launch_gather_u<T>((const V2<T>*)c->vbuf[0], (const V2<T>*)c->dbuf[0], (V2<T>*)c->ubuf[0], c->Lx, c->Ly, s);
  for (int bps : {2, 3, 4, 5, 6, 8, 16}) {
    double ms;
    if ((r = timeit([&] {
           cg::launch_heun<T>(c->st, sp, (const V2<T>*)c->vbuf[0], (const V2<T>*)c->vbuf[1],
                              (V2<T>*)c->dbuf[0], (V2<T>*)c->dbuf[1], (V2<T>*)c->ubuf[0], (V2<T>*)c->ubuf[1],
                              c->Lx, c->Ly, cg::kModeFixed, h, 0, 0, bps, s);
         }, &ms)))
      return r;
    if (ms < best_ms[2]) { best_ms[2] = ms; best.heun_bps = bps; }
  }
  CG_CUDA(c, cudaGetLastError());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->tune = best;
  for (int k = 0; k < 3; ++k) c->tune_ms[k] = best_ms[k];
  c->tuned = true;
  // graphs captured with other shapes are rebuilt on next use
  if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  drop_outer_graph(c);
  return CG_OK;
}

// attempts per body of the step loop's WHILE node (measured at 1024^2: 8 takes 1 % less
// time than 4, 16 no less than 8; the attempts after the last one return at once)
constexpr int kGraphUnroll = 8;
static_assert(kGraphUnroll % 2 == 0, "a body starts at an even attempt: the step loop state alternates slots");

// ---- graph capture ----------------------------------------------------------

// The graph that stream `s` is capturing into.
cudaError_t captured_graph(cudaStream_t s, cudaGraph_t* g) {
  cudaStreamCaptureStatus st;
  return cudaStreamGetCaptureInfo(s, &st, nullptr, g, nullptr, nullptr, nullptr);
}

// Append a conditional WHILE node (handle h) after the work captured so far on `cs`, and
// capture body(bs) into its body graph on the spare stream `bs`.
template <typename F>
cudaError_t capture_while(cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle h, F&& body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return e;
  const cudaError_t eb = body(bs);
  cudaGraph_t bg = nullptr;
  e = cudaStreamEndCapture(bs, &bg);
  return eb != cudaSuccess ? eb : e;
}

// One integration of the current spectrum: init kernels, then a WHILE node whose body
// is kGraphUnroll attempted steps (the kernels of an attempt after the integration has
// ended return at once; the init kernel sets the condition, the step controller clears
// it), then the snapshot of the projected grid into dres and the outcome into info.
template <typename T>
cudaError_t capture_integration(cg_ctx* c, cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle* hout) {
  cudaGraph_t g = nullptr;
  cudaError_t e = captured_graph(cs, &g);
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) return e;
  const bool lin = c->opt.flow == CG_FLOW_LINEAR;
  if (lin) enqueue_init_linear<T>(c, h, 1, cs);
  else enqueue_init<T>(c, h, 1, cs);
  e = capture_while(cs, bs, h, [&](cudaStream_t s) {
    for (int k = 0; k < kGraphUnroll; ++k) {
      if (lin) enqueue_body_linear<T>(c, h, 1, s);
      else enqueue_body<T>(c, h, 1, s, k);
    }
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  enqueue_finish<T>(c, cs);
  if (hout) *hout = h;
  return cudaGetLastError();
}

// The whole outer iteration of one context, captured on `cs` (a stream capturing into
// a graph; bs and bs2 are spare streams for the loop bodies): areas and the first
// decision, then a WHILE node whose body is one iteration.
template <typename T>
cudaError_t capture_cartogram(cg_ctx* c, cudaStream_t cs, cudaStream_t bs, cudaStream_t bs2) {
  cudaGraph_t g = nullptr;
  cudaError_t e = captured_graph(cs, &g);
  cudaGraphConditionalHandle ho = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, g, 0, 0);
  if (e != cudaSuccess) return e;
  cg::launch_areas(c->xy, c->ring_off, c->area_sums, c->reg_off, c->reg_rings, c->values, c->R_n,
                   c->area, c->err_d, c->w, c->info, area_chunks(c), cs);
  cg::launch_outer_decide(c->outer, c->info, ho, 0, cs);
  const int N = c->Lx * c->Ly;
  return capture_while(cs, bs, ho, [&](cudaStream_t s) {
    cudaError_t eb = cudaMemsetAsync(c->acc, 0, sizeof(double) * (size_t)N, s);
    if (eb != cudaSuccess) return eb;
    cg::launch_raster(c->xy, c->next, c->vreg, c->w, c->acc, c->Lx, c->Ly, (int)c->n_vert, s);
    cg::launch_blur_tables(c->outer, 0.0, c->bx, c->by, c->Lx, c->Ly, s);
    launch_forward<T>(c, c->bx, c->by, s);
    if ((eb = capture_integration<T>(c, s, bs2, nullptr)) != cudaSuccess) return eb;
    cg::launch_outer_commit<T>(c->outer, c->info, (const V2<T>*)c->dres, N, s);
    cg::launch_map_points<T>(c->xy, c->xy, c->n_vert, (const V2<T>*)c->dres, c->Lx, c->Ly, s, &c->outer->status);
    cg::launch_areas(c->xy, c->ring_off, c->area_sums, c->reg_off, c->reg_rings, c->values, c->R_n,
                     c->area, c->err_d, c->w, c->info, area_chunks(c), s);
    cg::launch_outer_decide(c->outer, c->info, ho, 1, s);
    return cudaGetLastError();
  });
}

// Capture `enqueue(cs, bs, bs2)` into a new graph and instantiate it.
template <typename F>
int capture_and_instantiate(cg_ctx* c, cudaGraph_t* gout, cudaGraphExec_t* xout, F&& enqueue) {
  cudaStream_t cs = nullptr, bs = nullptr, bs2 = nullptr;
  CG_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  CG_CUDA(c, cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  CG_CUDA(c, cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  int rc = CG_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    e = enqueue(cs, bs, bs2);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(xout, g, 0);
  if (e != cudaSuccess) {
    rc = fail(c, CG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    if (g) cudaGraphDestroy(g);
  } else {
    *gout = g;
  }
  cudaGetLastError();
  cudaStreamDestroy(cs);
  cudaStreamDestroy(bs);
  cudaStreamDestroy(bs2);
  return rc;
}

// Graph of one integration (cartogram_integrate_once, and the host-driven outer loop).
template <typename T>
int build_graph(cg_ctx* c) {
  return capture_and_instantiate(c, &c->graph, &c->exec, [&](cudaStream_t cs, cudaStream_t bs, cudaStream_t) {
    return capture_integration<T>(c, cs, bs, &c->cond);
  });
}

void drop_outer_graph(cg_ctx* c) {
  if (c->oexec) cudaGraphExecDestroy(c->oexec);
  if (c->ograph) cudaGraphDestroy(c->ograph);
  c->oexec = nullptr;
  c->ograph = nullptr;
  ++c->gen;
}

template <typename T>
int run_integration_host(cg_ctx* c);

// Run one integration of the current spectrum; the projected grid ends in dres and
// the outcome in info (device). Records the step-loop time between ev0 and ev1.
template <typename T>
int run_integration(cg_ctx* c) {
  cudaStream_t s = c->stream;
  if (c->opt.use_graph == 2 && c->persist_grid > 0 && c->opt.flow == CG_FLOW_DIFFUSION) {
    cg::IntegrateArgs<T> a;
    a.spec = (const T*)c->specT;
    a.ABt = (V2<T>*)c->AB;
    a.Wx = (const V2<T>*)c->Wx;
    a.Ex = (const V2<T>*)c->Ex;
    a.Wy = (const V2<T>*)c->Wy;
    a.Ey = (const V2<T>*)c->Ey;
    a.v0 = (V2<T>*)c->vbuf[0];
    a.v1 = (V2<T>*)c->vbuf[1];
    a.d0 = (V2<T>*)c->dbuf[0];
    a.d1 = (V2<T>*)c->dbuf[1];
    a.dres = (V2<T>*)c->dres;
    a.st = c->st;
    a.gb = c->gb;
    a.acc = c->acc2;
    a.sp = step_params(c);
    a.Lx = c->Lx;
    a.Ly = c->Ly;
    a.log2Lx = c->log2Lx;
    a.log2Ly = c->log2Ly;
    a.S = c->persist_rows;
    a.Wc = c->persist_cols;
    a.spins = c->opt.barrier_spins;
    CG_CUDA(c, cudaEventRecord(c->ev0, s));
    CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
    CG_CUDA(c, cudaMemsetAsync(c->gb, 0, sizeof(cg::GridBarrier), s));
    CG_CUDA(c, cudaMemsetAsync(c->acc2, 0, 2 * sizeof(cg::StepAcc), s));
    CG_CUDA(c, cg::launch_integrate<T>(a, c->persist_grid, c->persist_smem, s));
    cg::launch_collect(c->st, c->info, s);
    CG_CUDA(c, cudaEventRecord(c->ev1, s));
    return CG_OK;
  }
  if (c->opt.use_graph) {
    if (!c->exec) {
      int r = build_graph<T>(c);
      if (r) return r;
    }
    CG_CUDA(c, cudaEventRecord(c->ev0, s));
    CG_CUDA(c, cudaGraphLaunch(c->exec, s));
    CG_CUDA(c, cudaEventRecord(c->ev1, s));
    return CG_OK;
  }
  return run_integration_host<T>(c);
}

// One integration with the step loop driven from the host (the same kernels; the
// kernels of an attempt after the end return at once).
template <typename T>
int run_integration_host(cg_ctx* c) {
  cudaStream_t s = c->stream;
  CG_CUDA(c, cudaEventRecord(c->ev0, s));
  const bool lin = c->opt.flow == CG_FLOW_LINEAR;
  if (lin) enqueue_init_linear<T>(c, 0, 0, s);
  else enqueue_init<T>(c, 0, 0, s);
  const int chunk = 8;  // even: each chunk starts at an even attempt
  for (long long done = 0; done < (long long)c->opt.max_steps + chunk; done += chunk) {
    for (int k = 0; k < chunk; ++k) {
      if (lin) enqueue_body_linear<T>(c, 0, 0, s);
      else enqueue_body<T>(c, 0, 0, s, k);
    }
    cg::launch_collect(c->st, c->info, s);
    CG_CUDA(c, cudaMemcpyAsync(c->info_h, c->info, sizeof(IterInfo), cudaMemcpyDeviceToHost, s));
    CG_CUDA(c, cudaStreamSynchronize(s));
    if (c->info_h->status != cg::kRunning) break;
  }
  enqueue_finish<T>(c, s);
  CG_CUDA(c, cudaEventRecord(c->ev1, s));
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

template <typename T>
int run_forward(cg_ctx* c) {
  // blur width of this outer iteration: blur * decay^k
  const double sigma = c->blur * std::pow(c->opt.blur_decay, (double)c->hist_len);
  const bool blur = sigma > 0.0;
  if (blur && sigma != c->blur_tab_sigma) {
    int r = set_blur_tables(c, sigma);
    if (r) return r;
  }
  launch_forward<T>(c, blur ? c->bx : nullptr, blur ? c->by : nullptr, c->stream);
  c->have_spectrum = true;
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int run_raster(cg_ctx* c) {
  CG_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(double) * (size_t)c->Lx * c->Ly, c->stream));
  cg::launch_raster(c->xy, c->next, c->vreg, c->w, c->acc, c->Lx, c->Ly, (int)c->n_vert, c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int run_areas(cg_ctx* c) {
  cg::launch_areas(c->xy, c->ring_off, c->area_sums, c->reg_off, c->reg_rings,
                   c->values, c->R_n, c->area, c->err_d, c->w, c->info, area_chunks(c), c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int read_info(cg_ctx* c) {
  CG_CUDA(c, cudaMemcpyAsync(c->info_h, c->info, sizeof(IterInfo), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return CG_OK;
}

// The outer iteration driven by the host: one graph launch (or host loop) per
// integration, a read-back of the outcome and of the areas after each. Runs at most
// iter_limit iterations; stopping there is CG_ENOCONVERGE only when that is the whole
// budget (final), else *stopped is set. Counts accumulate into s.
// Bytes of one history slot: the projected grid's displacements, then its IterRecord.
template <typename T>
size_t slot_bytes(const cg_ctx* c) {
  return sizeof(V2<T>) * (size_t)c->Lx * c->Ly + sizeof(cg::IterRecord);
}

template <typename T>
int do_integrate_host(cg_ctx* c, cg_stats& s, int iter_limit, bool final, bool* stopped) {
  int r;
  if (stopped) *stopped = false;
  if ((r = run_areas(c)) || (r = read_info(c))) return r;
  double max_err = c->info_h->max_err;
  int status = CG_OK;
  const size_t fbytes = sizeof(V2<T>) * (size_t)c->Lx * c->Ly;
  const size_t sbytes = slot_bytes<T>(c);
  int it = 0;
  while (!(max_err < c->opt.area_tol)) {
    if (it >= iter_limit) {
      if (final)
        status = fail(c, CG_ENOCONVERGE, "no convergence after %d iterations (max error %g)", s.iterations + it,
                      max_err);
      else if (stopped)
        *stopped = true;
      break;
    }
    if ((r = run_raster(c)) || (r = run_forward<T>(c)) || (r = run_integration<T>(c)) ||
        (r = read_info(c)))
      return r;
    const IterInfo inf = *c->info_h;
    float ms = 0.f;
    CG_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    s.step_loop_ms += ms;
    s.steps_accepted += inf.accepted;
    s.steps_rejected += inf.rejected;
    s.t_end = inf.t_end;
    if (inf.status != cg::kDone) {
      status = fail(c, inf.status == cg::kTimeout ? CG_ETIMEOUT : CG_ESTEPFAIL,
                    "integration %d ended with status %d after %lld/%lld steps", s.iterations + it + 1,
                    inf.status, inf.accepted, inf.rejected);
      break;
    }
    // pick the launch shapes once, on the displacements of a real integration
    if (c->opt.autotune && !c->tuned && (r = do_autotune<T>(c, 10))) return r;
    if ((int)c->hist.size() <= c->hist_len) {
      void* p = nullptr;
      CG_CUDA(c, cudaMalloc(&p, sbytes));
      c->hist.push_back(p);
    }
    void* grid = c->hist[c->hist_len];
    CG_CUDA(c, cudaMemcpyAsync(grid, c->dres, fbytes, cudaMemcpyDeviceToDevice, c->stream));
    cg::launch_map_points<T>(c->xy, c->xy, c->n_vert, (const V2<T>*)grid, c->Lx, c->Ly, c->stream);
    if ((r = run_areas(c)) || (r = read_info(c))) return r;
    max_err = c->info_h->max_err;
    cg::IterRecord rec;
    rec.max_err = max_err;
    rec.t_end = inf.t_end;
    rec.blur = c->blur * std::pow(c->opt.blur_decay, (double)c->hist_len);
    rec.accepted = inf.accepted;
    rec.rejected = inf.rejected;
    rec.loop_ns = inf.loop_ns;
    CG_CUDA(c, cudaMemcpy(static_cast<char*>(grid) + fbytes, &rec, sizeof rec, cudaMemcpyHostToDevice));
    ++it;
    ++c->hist_len;
  }
  s.iterations += it;
  s.max_area_error = max_err;
  return status;
}

// Host side of a device-run outer iteration: history slots for the coming iterations
// (in chunks), the slot pointers and blur widths on the device, the loop state.
constexpr int kSlotChunk = 32;

template <typename T>
int ensure_slots(cg_ctx* c, int want) {
  const size_t sbytes = slot_bytes<T>(c);
  while ((int)c->hist.size() < want) {
    void* p = nullptr;
    CG_CUDA(c, cudaMalloc(&p, sbytes));
    c->hist.push_back(p);
  }
  const int n = (int)c->hist.size();
  if (n == c->hist_d_count) return CG_OK;
  if (c->hist_d_cap < n) {
    if (c->hist_d) CG_CUDA(c, cudaFree(c->hist_d));
    c->hist_d = nullptr;
    c->hist_d_cap = std::max(n, 2 * c->hist_d_cap);
    CG_CUDA(c, cudaMalloc((void**)&c->hist_d, sizeof(void*) * c->hist_d_cap));
  }
  CG_CUDA(c, cudaMemcpy(c->hist_d, c->hist.data(), sizeof(void*) * n, cudaMemcpyHostToDevice));
  c->hist_d_count = n;
  return CG_OK;
}

// Prepare one context's device loop for up to `budget` iterations: blur widths of those
// iterations, the first chunk of slots, the loop state (written to the device on the
// context's stream).
template <typename T>
int outer_prepare(cg_ctx* c, int budget) {
  if (c->sigma_cap < budget + 1) {
    if (c->sigma_d) CG_CUDA(c, cudaFree(c->sigma_d));
    if (c->sigma_h) CG_CUDA(c, cudaFreeHost(c->sigma_h));
    c->sigma_d = nullptr;
    c->sigma_h = nullptr;
    c->sigma_cap = budget + 1;
    CG_CUDA(c, cudaMalloc((void**)&c->sigma_d, sizeof(double) * c->sigma_cap));
    CG_CUDA(c, cudaMallocHost((void**)&c->sigma_h, sizeof(double) * c->sigma_cap));
  }
  CG_CUDA(c, cudaStreamSynchronize(c->stream));  // the pinned staging is free
  for (int i = 0; i <= budget; ++i)
    c->sigma_h[i] = c->blur * std::pow(c->opt.blur_decay, (double)(c->hist_len + i));
  CG_CUDA(c, cudaMemcpyAsync(c->sigma_d, c->sigma_h, sizeof(double) * (budget + 1), cudaMemcpyHostToDevice,
                             c->stream));
  int r = ensure_slots<T>(c, c->hist_len + std::min(budget, kSlotChunk));
  if (r) return r;
  cg::OuterState& o = *c->outer_h;
  memset(&o, 0, sizeof o);
  o.hist = c->hist_d;
  o.sigma = c->sigma_d;
  o.area_tol = c->opt.area_tol;
  o.k = c->hist_len;
  o.cap = (int)c->hist.size();
  o.iterations = 0;
  o.max_iter = budget;
  o.status = cg::kOuterRunning;
  o.rec_offset = sizeof(V2<T>) * (size_t)c->Lx * c->Ly;
  CG_CUDA(c, cudaMemcpyAsync(c->outer, &o, sizeof o, cudaMemcpyHostToDevice, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->blur_tab_sigma = -1.0;  // the loop rewrites the blur tables
  return CG_OK;
}

// After a device loop stopped for want of slots: add a chunk and resume.
template <typename T>
int outer_resume(cg_ctx* c) {
  cg::OuterState& o = *c->outer_h;
  const int left = o.max_iter - o.iterations;
  int r = ensure_slots<T>(c, o.k + std::min(left, kSlotChunk));
  if (r) return r;
  o.hist = c->hist_d;
  o.cap = (int)c->hist.size();
  o.status = cg::kOuterRunning;
  CG_CUDA(c, cudaMemcpy(c->outer, &o, sizeof o, cudaMemcpyHostToDevice));
  return CG_OK;
}

// Fold a finished device loop into the context and the statistics.
int outer_finish(cg_ctx* c, cg_stats& s) {
  const cg::OuterState& o = *c->outer_h;
  c->hist_len = o.k;
  if (o.iterations > 0 || o.accepted + o.rejected > 0) c->have_spectrum = true;
  s.iterations += o.iterations;
  s.steps_accepted += o.accepted;
  s.steps_rejected += o.rejected;
  if (o.accepted + o.rejected > 0) s.t_end = o.t_end;
  s.step_loop_ms += o.loop_ns * 1e-6;
  s.max_area_error = o.max_err;
  if (o.status == cg::kOuterConverged) return CG_OK;
  if (o.status == cg::kOuterNoConverge)
    return fail(c, CG_ENOCONVERGE, "no convergence after %d iterations (max error %g)", s.iterations, o.max_err);
  return fail(c, o.status == cg::kTimeout ? CG_ETIMEOUT : CG_ESTEPFAIL,
              "integration %d ended with status %d", s.iterations + 1, o.status);
}

template <typename T>
int build_outer_graph(cg_ctx* c) {
  return capture_and_instantiate(c, &c->ograph, &c->oexec, [&](cudaStream_t cs, cudaStream_t bs, cudaStream_t bs2) {
    return capture_cartogram<T>(c, cs, bs, bs2);
  });
}

// First iteration on the host path when the launch shapes are still to be picked (on
// the displacements of a real integration). Returns CG_OK with *go = true when the
// device loop should continue.
template <typename T>
int maybe_tune_first(cg_ctx* c, cg_stats& s, bool* go) {
  *go = true;
  if (!c->opt.autotune || c->tuned || c->opt.max_iter == 0) return CG_OK;
  bool stopped = false;
  const int r = do_integrate_host<T>(c, s, 1, c->opt.max_iter == 1, &stopped);
  *go = r == CG_OK && stopped;
  return r;
}

// The outer iteration run on the device: one launch of the context's cartogram graph,
// again only when history slots ran out.
template <typename T>
int do_integrate_device(cg_ctx* c, cg_stats& s) {
  bool go = false;
  int r = maybe_tune_first<T>(c, s, &go);
  if (r || !go) return r;
  if (!c->oexec && (r = build_outer_graph<T>(c))) return r;
  if ((r = outer_prepare<T>(c, c->opt.max_iter - s.iterations))) return r;
  for (;;) {
    CG_CUDA(c, cudaGraphLaunch(c->oexec, c->stream));
    CG_CUDA(c, cudaMemcpyAsync(c->outer_h, c->outer, sizeof(cg::OuterState), cudaMemcpyDeviceToHost, c->stream));
    CG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->outer_h->status != cg::kOuterNeedSlots) break;
    if ((r = outer_resume<T>(c))) return r;
  }
  return outer_finish(c, s);
}

template <typename T>
int do_integrate(cg_ctx* c, cg_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  cg_stats s;
  memset(&s, 0, sizeof s);
  int status;
  stamp_deadline(c);
  if (c->opt.use_graph == 1) status = do_integrate_device<T>(c, s);
  else status = do_integrate_host<T>(c, s, c->opt.max_iter, true, nullptr);
  s.converged = s.max_area_error < c->opt.area_tol;
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = s;
  return status;
}

bool is_finite(double v) { return std::isfinite(v); }

int check_ctx(cg_ctx* c, bool need_regions) {
  if (!c) return CG_EINVAL;
  c->err.clear();
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, CG_ECUDA, "cudaSetDevice failed");
  if (need_regions && !c->have_regions) return fail(c, CG_ESTATE, "no map: call cartogram_set_regions first");
  return CG_OK;
}

template <typename T>
int copy_field_out(cg_ctx* c, const void* src, double* dst, int comps) {
  // widen T -> double on the host (entry points for inspection, not the hot path)
  const size_t n = (size_t)c->Lx * c->Ly * comps;
  std::vector<T> h(n);
  CG_CUDA(c, cudaMemcpyAsync(h.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<double> o(h.begin(), h.end());
  CG_CUDA(c, cudaMemcpy(dst, o.data(), sizeof(double) * n, cudaMemcpyDefault));
  return CG_OK;
}

template <typename T>
int copy_field_in(cg_ctx* c, const double* src, void* dst, int comps) {
  const size_t n = (size_t)c->Lx * c->Ly * comps;
  std::vector<double> h(n);
  CG_CUDA(c, cudaMemcpy(h.data(), src, sizeof(double) * n, cudaMemcpyDefault));
  std::vector<T> t(h.begin(), h.end());
  CG_CUDA(c, cudaMemcpyAsync(dst, t.data(), sizeof(T) * n, cudaMemcpyHostToDevice, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return CG_OK;
}

template <typename T>
int do_velocity(cg_ctx* c, double t, double* rho_out, double* v_out) {
  CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  enqueue_field<T>(c, cg::kModeFixed, t, (V2<T>*)c->vbuf[0], (V2<T>*)c->vbuf[1], (T*)c->rho_tmp,
                   c->stream);
  CG_CUDA(c, cudaGetLastError());
  int r;
  if (rho_out && (r = copy_field_out<T>(c, c->rho_tmp, rho_out, 1))) return r;
  if (v_out && (r = copy_field_out<T>(c, c->vbuf[0], v_out, 2))) return r;
  return CG_OK;
}

template <typename T>
int do_heun(cg_ctx* c, double t, double h, const double* din, double* dout, double* err) {
  CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  enqueue_field<T>(c, cg::kModeFixed, t, (V2<T>*)c->vbuf[0], nullptr, nullptr, c->stream);
  enqueue_field<T>(c, cg::kModeFixed, t + h, (V2<T>*)c->vbuf[1], nullptr, nullptr, c->stream);
  int r = copy_field_in<T>(c, din, c->dbuf[0], 2);
  if (r) return r;
  CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  // the step loop's kernel: predictor velocities gathered once, then read from the cache
  cg::launch_gather_u<T>((const V2<T>*)c->vbuf[0], (const V2<T>*)c->dbuf[0], (V2<T>*)c->ubuf[0], c->Lx, c->Ly,
                         c->stream);
  cg::launch_heun<T>(c->st, step_params(c), (const V2<T>*)c->vbuf[0], (const V2<T>*)c->vbuf[1],
                     (V2<T>*)c->dbuf[0], (V2<T>*)c->dbuf[1], (V2<T>*)c->ubuf[0], (V2<T>*)c->ubuf[1], c->Lx,
                     c->Ly, cg::kModeFixed, h, 0, 0, c->tune.heun_bps, c->stream);
  CG_CUDA(c, cudaGetLastError());
  if ((r = copy_field_out<T>(c, c->dbuf[1], dout, 2))) return r;
  DevState hs;
  CG_CUDA(c, cudaMemcpy(&hs, c->st, sizeof hs, cudaMemcpyDeviceToHost));
  if (err) {
    double e2;
    memcpy(&e2, &hs.err2_bits, sizeof e2);
    *err = std::sqrt(e2);
  }
  return CG_OK;
}

template <typename T>
int grid_out(cg_ctx* c, const void* disp, double* out) {
  const size_t N = (size_t)c->Lx * c->Ly;
  std::vector<T> h(2 * N);
  CG_CUDA(c, cudaMemcpyAsync(h.data(), disp, sizeof(T) * 2 * N, cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<double> o(2 * N);
  for (int j = 0; j < c->Ly; ++j)
    for (int i = 0; i < c->Lx; ++i) {
      const size_t p = (size_t)j * c->Lx + i;
      o[2 * p] = i + 0.5 + (double)h[2 * p];
      o[2 * p + 1] = j + 0.5 + (double)h[2 * p + 1];
    }
  CG_CUDA(c, cudaMemcpy(out, o.data(), sizeof(double) * 2 * N, cudaMemcpyDefault));
  return CG_OK;
}

template <typename T>
int do_integrate_once(cg_ctx* c, double* grid, long long* acc, long long* rej, double* t_end) {
  stamp_deadline(c, false);  // the time limit is for cartogram_integrate and batches
  int r = run_integration<T>(c);
  if (r) return r;
  if ((r = read_info(c))) return r;
  const IterInfo inf = *c->info_h;
  if (acc) *acc = inf.accepted;
  if (rej) *rej = inf.rejected;
  if (t_end) *t_end = inf.t_end;
  if (grid && (r = grid_out<T>(c, c->dres, grid))) return r;
  if (inf.status != cg::kDone)
    return fail(c, inf.status == cg::kTimeout ? CG_ETIMEOUT : CG_ESTEPFAIL, "integration ended with status %d",
                inf.status);
  return CG_OK;
}

int ensure_pts(cg_ctx* c, long long n) {
  if (n > c->pts_cap) {
    if (c->pts) cudaFree(c->pts);
    c->pts = nullptr;
    c->pts_cap = 0;
    CG_CUDA(c, cudaMalloc((void**)&c->pts, sizeof(double2) * n));
    c->pts_cap = n;
  }
  return CG_OK;
}

template <typename T>
int do_project(cg_ctx* c, int64_t n, const double* in, double* out) {
  if (n == 0) return CG_OK;
  int r = ensure_pts(c, n);
  if (r) return r;
  CG_CUDA(c, cudaMemcpyAsync(c->pts, in, sizeof(double2) * n, cudaMemcpyDefault, c->stream));
  for (int k = 0; k < c->hist_len; ++k)
    cg::launch_map_points<T>(c->pts, c->pts, n, (const V2<T>*)c->hist[k], c->Lx, c->Ly, c->stream);
  CG_CUDA(c, cudaGetLastError());
  CG_CUDA(c, cudaMemcpyAsync(out, c->pts, sizeof(double2) * n, cudaMemcpyDefault, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return CG_OK;
}

// The first hist_len history slots as a device pointer table.
template <typename T>
int hist_table(cg_ctx* c) {
  return ensure_slots<T>(c, (int)c->hist.size());
}

template <typename T>
int do_distortion(cg_ctx* c, double* out) {
  int r = hist_table<T>(c);
  if (r) return r;
  if (!c->diag) {
    const int nb = cg::distortion_blocks(c->Lx, c->Ly);
    CG_CUDA(c, cudaMalloc((void**)&c->diag, sizeof(double) * (2 * nb + 8)));
  }
  const int nb = cg::distortion_blocks(c->Lx, c->Ly);
  double* part = c->diag;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(c->diag + 2 * nb);
  double* res = c->diag + 2 * nb + 2;
  cg::launch_distortion<T>((const void* const*)c->hist_d, c->hist_len, c->Lx, c->Ly, part, mx, res, c->stream);
  CG_CUDA(c, cudaGetLastError());
  double h[4];
  CG_CUDA(c, cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  CG_CUDA(c, cudaMemcpy(out, h, sizeof h, cudaMemcpyDefault));
  return CG_OK;
}

template <typename T>
int do_inverse_project(cg_ctx* c, int64_t n, const double* in, double* out) {
  if (n == 0) return CG_OK;
  int r = hist_table<T>(c);
  if (r || (r = ensure_pts(c, n))) return r;
  CG_CUDA(c, cudaMemcpyAsync(c->pts, in, sizeof(double2) * n, cudaMemcpyDefault, c->stream));
  cg::launch_inverse_points<T>((const void* const*)c->hist_d, c->hist_len, c->Lx, c->Ly, n, c->pts, c->stream);
  CG_CUDA(c, cudaGetLastError());
  CG_CUDA(c, cudaMemcpyAsync(out, c->pts, sizeof(double2) * n, cudaMemcpyDefault, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return CG_OK;
}

// ---- gradient of one outer iteration (FP64) -----------------------------------

void free_adj(cg_ctx* c) {
  AdjWork* a = c->adj;
  if (!a) return;
  std::vector<void*> ps = {a->Dk, a->lam, a->L[0], a->L[1], a->a_rho, a->a_gx, a->a_gy, a->Crho, a->Cx, a->Cy,
                           a->lam_spec, a->specp, a->R, a->dens, a->AB, a->flux, a->sched, a->vals, a->dLdA,
                           a->gw, a->dsig, a->xy1, a->gv, a->gv2, a->R2[0], a->R2[1], a->AB2[0], a->AB2[1]};
  for (auto p : a->X) ps.push_back(p);
  for (auto p : a->spec) ps.push_back(p);
  for (auto p : a->v) ps.push_back(p);
  for (auto p : a->rho) ps.push_back(p);
  for (auto p : a->D) ps.push_back(p);
  for (auto p : a->ckpt) ps.push_back(p);
  for (void* p : ps)
    if (p) cudaFree(p);
  for (int k = 0; k < 2; ++k) {
    if (a->side[k]) cudaStreamDestroy(a->side[k]);
    if (a->join[k]) cudaEventDestroy(a->join[k]);
  }
  if (a->fork) cudaEventDestroy(a->fork);
  delete a;
  c->adj = nullptr;
}

int adj_alloc(cg_ctx* c, int C) {
  if (c->adj && c->adj->C == C) return CG_OK;
  free_adj(c);
  AdjWork* a = new AdjWork();
  c->adj = a;
  a->C = C;
  const size_t N = (size_t)c->Lx * c->Ly;
  CG_CUDA(c, cudaMalloc((void**)&a->lam, sizeof(double2) * N));
  for (int k = 0; k < 2; ++k) CG_CUDA(c, cudaMalloc((void**)&a->L[k], sizeof(double) * 2 * N));
  double** ds[] = {&a->a_rho, &a->a_gx, &a->a_gy, &a->Crho, &a->Cx, &a->Cy, &a->lam_spec, &a->specp, &a->R, &a->dens};
  for (double** p : ds) CG_CUDA(c, cudaMalloc((void**)p, sizeof(double) * N));
  CG_CUDA(c, cudaMalloc((void**)&a->AB, sizeof(double2) * N));
  for (int k = 0; k < 2; ++k) {
    CG_CUDA(c, cudaMalloc((void**)&a->R2[k], sizeof(double) * N));
    CG_CUDA(c, cudaMalloc((void**)&a->AB2[k], sizeof(double2) * N));
    CG_CUDA(c, cudaStreamCreateWithFlags(&a->side[k], cudaStreamNonBlocking));
    CG_CUDA(c, cudaEventCreateWithFlags(&a->join[k], cudaEventDisableTiming));
  }
  CG_CUDA(c, cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming));
  CG_CUDA(c, cudaMalloc((void**)&a->Dk, sizeof(double2) * N));
  CG_CUDA(c, cudaMalloc((void**)&a->flux, sizeof(double2) * N));
  a->v.assign(C + 1, nullptr);
  a->rho.assign(C + 1, nullptr);
  a->D.assign(C + 1, nullptr);
  for (int k = 0; k <= C; ++k) {
    CG_CUDA(c, cudaMalloc((void**)&a->v[k], sizeof(double2) * N));
    CG_CUDA(c, cudaMalloc((void**)&a->rho[k], sizeof(double) * N));
    CG_CUDA(c, cudaMalloc((void**)&a->D[k], sizeof(double2) * N));
  }
  CG_CUDA(c, cudaMalloc((void**)&a->sched, sizeof(double) * 2 * (size_t)c->opt.max_steps));
  a->n_regions = c->R_n;
  a->n_vert = c->n_vert;
  CG_CUDA(c, cudaMalloc((void**)&a->vals, sizeof(double) * c->R_n));
  CG_CUDA(c, cudaMalloc((void**)&a->dLdA, sizeof(double) * c->R_n));
  CG_CUDA(c, cudaMalloc((void**)&a->gw, sizeof(double) * c->R_n));
  CG_CUDA(c, cudaMalloc((void**)&a->dsig, sizeof(double)));
  CG_CUDA(c, cudaMalloc((void**)&a->xy1, sizeof(double2) * std::max<long long>(1, c->n_vert)));
  CG_CUDA(c, cudaMalloc((void**)&a->gv, sizeof(double2) * std::max<long long>(1, c->n_vert)));
  CG_CUDA(c, cudaMalloc((void**)&a->gv2, sizeof(double2) * std::max<long long>(1, c->n_vert)));
  return CG_OK;
}

// Per-iteration storage of a K-iteration gradient.
int adj_alloc_iters(cg_ctx* c, int K) {
  AdjWork* a = c->adj;
  const size_t N = (size_t)c->Lx * c->Ly;
  while ((int)a->X.size() < K + 1) {
    double2* p = nullptr;
    CG_CUDA(c, cudaMalloc((void**)&p, sizeof(double2) * std::max<long long>(1, c->n_vert)));
    a->X.push_back(p);
  }
  while ((int)a->spec.size() < K) {
    double* p = nullptr;
    CG_CUDA(c, cudaMalloc((void**)&p, sizeof(double) * N));
    a->spec.push_back(p);
  }
  return CG_OK;
}

// Field v (and density) of the FP64 path at time tau, from the iteration's spectrum.
void adj_field(cg_ctx* c, double tau, double2* v, double* rho, double2* AB = nullptr, cudaStream_t s = nullptr) {
  AdjWork* a = c->adj;
  if (!AB) AB = a->AB;
  if (!s) s = c->stream;
  cg::launch_inv_rows<double>(c->log2Lx, c->Ly, c->tune.rows, c->spec64, AB, (const double2*)c->Wx,
                              (const double2*)c->Ex, c->st, cg::kModeFixed, tau, 0, 0, 0u, s);
  cg::launch_inv_cols<double>(c->log2Ly, c->Lx, c->tune.cols, AB, v, nullptr, rho, (const double2*)c->Wy,
                              (const double2*)c->Ey, c->st, cg::kModeFixed, s);
}

// The fields of levels n0 .. n0 + m (times from the schedule) into v[0 .. m], rho[0 .. m]:
// they depend on the spectrum alone, so they run on three streams side by side (each FP64
// transform pair fills a fraction of the GPU at these sizes).
double adj_tau(const std::vector<double>& sch, int n);
void adj_fields(cg_ctx* c, const std::vector<double>& sch, int n0, int m) {
  AdjWork* a = c->adj;
  cudaStream_t s = c->stream;
  cudaEventRecord(a->fork, s);
  for (int q = 0; q < 2; ++q) cudaStreamWaitEvent(a->side[q], a->fork, 0);
  for (int k = 0; k <= m; ++k) {
    const int q = k % 3;
    adj_field(c, adj_tau(sch, n0 + k), a->v[k], a->rho[k], q ? a->AB2[q - 1] : a->AB, q ? a->side[q - 1] : s);
  }
  for (int q = 0; q < 2; ++q) {
    cudaEventRecord(a->join[q], a->side[q]);
    cudaStreamWaitEvent(s, a->join[q], 0);
  }
}

// One predictor-corrector step of all points with the fixed step h (the step kernel).
void adj_step(cg_ctx* c, const double2* v0, const double2* v1, const double2* din, double2* dout, double h) {
  cg::launch_heun<double>(c->st, step_params(c), v0, v1, (double2*)din, dout, nullptr, nullptr, c->Lx, c->Ly,
                          cg::kModeFixed, h, 0,
                          0, c->tune.heun_bps, c->stream);
}

// Level times of the schedule: tau_0 = 0, tau_{n+1} = tau_n + h_n (the device's sums).
double adj_tau(const std::vector<double>& sch, int n) {
  const int N = (int)sch.size() / 2;
  if (n < N) return sch[2 * n];
  return sch[2 * (N - 1)] + sch[2 * (N - 1) + 1];
}

// Process one time level's field adjoint: through v = -g/rho and the transposed
// transforms into the spectrum adjoint; clears the level's buffer.
void adj_level(cg_ctx* c, double* L, const double2* v, const double* rho, double tau) {
  AdjWork* a = c->adj;
  cudaStream_t s = c->stream;
  cg::launch_node_adjoint(L, v, rho, a->a_rho, a->a_gx, a->a_gy, c->Lx, c->Ly, s);
  double* ins[3] = {a->a_rho, a->a_gx, a->a_gy};
  double* outs[3] = {a->Crho, a->Cx, a->Cy};
  double* mid[3] = {a->R, a->R2[0], a->R2[1]};
  cudaStream_t on[3] = {s, a->side[0], a->side[1]};
  cudaEventRecord(a->fork, s);
  for (int k = 1; k < 3; ++k) cudaStreamWaitEvent(on[k], a->fork, 0);
  for (int k = 0; k < 3; ++k)
    cg::launch_fwd<double>(c->log2Lx, c->log2Ly, ins[k], mid[k], outs[k], nullptr, c->Wfx, c->Efx, c->Wfy, c->Efy,
                           nullptr, nullptr, on[k]);
  for (int k = 1; k < 3; ++k) {
    cudaEventRecord(a->join[k - 1], on[k]);
    cudaStreamWaitEvent(s, a->join[k - 1], 0);
  }
  cg::launch_spec_accumulate(a->Crho, a->Cx, a->Cy, a->lam_spec, tau, c->Lx, c->Ly, s);
  cudaMemsetAsync(L, 0, sizeof(double) * 2 * (size_t)c->Lx * c->Ly, s);
}

// Forward replay of one integration from the spectrum in spec64 with schedule sch:
// positions every C steps into the checkpoints (if ck), the final displacements returned.
double2* adj_replay(cg_ctx* c, const std::vector<double>& sch, int C, bool ck) {
  AdjWork* a = c->adj;
  cudaStream_t s = c->stream;
  const size_t N = (size_t)c->Lx * c->Ly;
  const int NS = (int)sch.size() / 2;
  if (ck) cudaMemsetAsync(a->ckpt[0], 0, sizeof(double2) * N, s);
  cudaMemsetAsync(a->D[0], 0, sizeof(double2) * N, s);
  double2* din = a->D[0];
  double2* dout = a->D[1];
  if (C >= 4) {
    // chunks of C steps: the chunk's C + 1 fields side by side, then its steps in order
    for (int n0 = 0; n0 < NS; n0 += C) {
      const int n1 = std::min(n0 + C, NS);
      adj_fields(c, sch, n0, n1 - n0);
      for (int n = n0; n < n1; ++n) {
        adj_step(c, a->v[n - n0], a->v[n - n0 + 1], din, dout, sch[2 * n + 1]);
        std::swap(din, dout);
        if (ck && (n + 1) % C == 0 && (n + 1) / C < (int)a->ckpt.size())
          cudaMemcpyAsync(a->ckpt[(n + 1) / C], din, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
      }
    }
    return din;
  }
  int cur = 0;  // v[cur] holds the field of level n
  adj_field(c, 0.0, a->v[0], a->rho[0]);
  for (int n = 0; n < NS; ++n) {
    adj_field(c, adj_tau(sch, n + 1), a->v[1 - cur], a->rho[1 - cur]);
    adj_step(c, a->v[cur], a->v[1 - cur], din, dout, sch[2 * n + 1]);
    std::swap(din, dout);
    cur = 1 - cur;
    if (ck && (n + 1) % C == 0 && (n + 1) / C < (int)a->ckpt.size())
      cudaMemcpyAsync(a->ckpt[(n + 1) / C], din, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
  }
  return din;
}

// Reverse of one integration: a->lam holds the final displacements' adjoint on entry;
// the spectrum adjoint accumulates into lam_spec (zeroed here).
void adj_reverse(cg_ctx* c, const std::vector<double>& sch, int C) {
  AdjWork* a = c->adj;
  cudaStream_t s = c->stream;
  const size_t N = (size_t)c->Lx * c->Ly;
  const int NS = (int)sch.size() / 2;
  cudaMemsetAsync(a->lam_spec, 0, sizeof(double) * N, s);
  cudaMemsetAsync(a->L[0], 0, sizeof(double) * 2 * N, s);
  cudaMemsetAsync(a->L[1], 0, sizeof(double) * 2 * N, s);
  // backwards over the segments; L[hi] holds level n + 1, L[lo] level n
  int hi = 0, lo = 1;
  const int nseg = (NS + C - 1) / C;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int n0 = sg * C, n1 = std::min(n0 + C, NS);
    cudaMemcpyAsync(a->D[0], a->ckpt[sg], sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
    adj_fields(c, sch, n0, n1 - n0);
    for (int k = 0; k < n1 - n0 - 1; ++k) adj_step(c, a->v[k], a->v[k + 1], a->D[k], a->D[k + 1], sch[2 * (n0 + k) + 1]);
    for (int n = n1 - 1; n >= n0; --n) {
      const int k = n - n0;
      cg::launch_heun_adjoint(a->D[k], a->v[k], a->v[k + 1], sch[2 * n + 1], a->lam, a->L[lo], a->L[hi], c->Lx,
                              c->Ly, s);
      adj_level(c, a->L[hi], a->v[k + 1], a->rho[k + 1], adj_tau(sch, n + 1));
      std::swap(hi, lo);
    }
  }
  // level 0 (its field is the first segment's level 0, still in place)
  if (NS > 0) adj_level(c, a->L[hi], a->v[0], a->rho[0], 0.0);
}

// A caller's own loss of the mapped vertices X' and areas A': its adjoints dL/dX' and
// dL/dA' (either may be NULL: zero) replace the built-in loss, and X', A' are returned.
struct Upstream {
  bool custom = false;
  const double* g_xy = nullptr;    // [n_vert][2]
  const double* g_area = nullptr;  // [R]
  double* xy_out = nullptr;        // [n_vert][2]
  double* area_out = nullptr;      // [R]
};

int do_iteration_gradient(cg_ctx* c, const double* values_in, double blur, double lam, int K, int replay, int C,
                          double* loss_out, double* grad_values, double* grad_blur,
                          const Upstream& up = Upstream()) {
  cudaStream_t s = c->stream;
  const int R = c->R_n;
  const size_t N = (size_t)c->Lx * c->Ly;
  const int nv = (int)c->n_vert;
  stamp_deadline(c, false);  // the time limit is for cartogram_integrate and batches
  std::vector<double> V(R);
  CG_CUDA(c, cudaMemcpy(V.data(), values_in, sizeof(double) * R, cudaMemcpyDefault));
  for (int i = 0; i < R; ++i)
    if (!is_finite(V[i]) || !(V[i] > 0.0)) return fail(c, CG_EINVAL, "value %d is not positive and finite", i);
  if (replay && (int)c->scheds.size() != K)
    return fail(c, CG_ESTATE, "no recorded schedule of %d iterations: call with replay = 0 first", K);
  int r = adj_alloc(c, C);
  if (r || (r = adj_alloc_iters(c, K))) return r;
  AdjWork* a = c->adj;
  CG_CUDA(c, cudaMemcpyAsync(a->vals, V.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
  CG_CUDA(c, cudaMemcpyAsync(a->X[0], c->xy, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, s));
  double sV = 0.0;
  for (int i = 0; i < R; ++i) sV += V[i];
  std::vector<std::vector<double>> A(K, std::vector<double>(R));
  std::vector<double> sigma(K), decay(K);
  if (!replay) c->scheds.assign(K, std::vector<double>());
  double2* D_last = nullptr;
  // forward: K outer iterations from the current vertices
  for (int k = 0; k < K; ++k) {
    decay[k] = std::pow(c->opt.blur_decay, (double)(c->hist_len + k));
    sigma[k] = blur * decay[k];
    cg::launch_areas(a->X[k], c->ring_off, c->area_sums, c->reg_off, c->reg_rings, a->vals, R,
                     c->area, c->err_d, c->w, c->info, area_chunks(c), s);
    CG_CUDA(c, cudaMemcpyAsync(A[k].data(), c->area, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    CG_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(double) * N, s));
    cg::launch_raster(a->X[k], c->next, c->vreg, c->w, c->acc, c->Lx, c->Ly, nv, s);
    cg::launch_blur_tables(nullptr, sigma[k], c->bx, c->by, c->Lx, c->Ly, s);
    cg::launch_fwd<double>(c->log2Lx, c->log2Ly, c->acc, c->R, c->spec64, nullptr, c->Wfx, c->Efx, c->Wfy, c->Efy,
                           c->bx, c->by, s);
    CG_CUDA(c, cudaMemcpyAsync(a->spec[k], c->spec64, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CG_CUDA(c, cudaGetLastError());
    if (!replay) {
      // the step schedule of an adaptive integration
      c->sched_rec = a->sched;
      r = run_integration_host<double>(c);
      c->sched_rec = nullptr;
      if (r || (r = read_info(c))) return r;
      const IterInfo inf = *c->info_h;
      if (inf.status != cg::kDone)
        return fail(c, inf.status == cg::kTimeout ? CG_ETIMEOUT : CG_ESTEPFAIL,
                    "integration %d ended with status %d after %lld/%lld steps", k + 1, inf.status, inf.accepted,
                    inf.rejected);
      c->scheds[k].assign(2 * (size_t)inf.accepted, 0.0);
      if (inf.accepted > 0)
        CG_CUDA(c, cudaMemcpy(c->scheds[k].data(), a->sched, sizeof(double) * 2 * inf.accepted,
                              cudaMemcpyDeviceToHost));
    }
    const int nck = (int)c->scheds[k].size() / 2 / C + 1;
    while ((int)a->ckpt.size() < nck) {
      double2* p = nullptr;
      CG_CUDA(c, cudaMalloc((void**)&p, sizeof(double2) * N));
      a->ckpt.push_back(p);
    }
    // the last iteration's replay keeps its checkpoints for the reverse pass
    double2* Dk = adj_replay(c, c->scheds[k], C, k == K - 1);
    if (k == K - 1) D_last = Dk;
    cg::launch_map_points<double>(a->X[k], a->X[k + 1], nv, Dk, c->Lx, c->Ly, s);
    CG_CUDA(c, cudaGetLastError());
  }
  c->have_spectrum = true;
  c->blur_tab_sigma = -1.0;
  // the loss on the final vertices
  cg::launch_areas(a->X[K], c->ring_off, c->area_sums, c->reg_off, c->reg_rings, a->vals, R, c->area,
                   c->err_d, c->w, c->info, area_chunks(c), s);
  std::vector<double> A1(R);
  std::vector<double2> X0(nv), X1(nv);
  CG_CUDA(c, cudaMemcpyAsync(A1.data(), c->area, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  CG_CUDA(c, cudaMemcpyAsync(X1.data(), a->X[K], sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
  CG_CUDA(c, cudaMemcpyAsync(X0.data(), a->X[0], sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
  CG_CUDA(c, cudaStreamSynchronize(s));
  if (up.custom) {
    if (up.xy_out) CG_CUDA(c, cudaMemcpy(up.xy_out, X1.data(), sizeof(double2) * nv, cudaMemcpyDefault));
    if (up.area_out) CG_CUDA(c, cudaMemcpy(up.area_out, A1.data(), sizeof(double) * R, cudaMemcpyDefault));
  }
  double sA1 = 0.0;
  for (int i = 0; i < R; ++i) sA1 += A1[i];
  std::vector<double> res(R);
  double L = 0.0, sres = 0.0;
  for (int i = 0; i < R && !up.custom; ++i) {
    if (!(A1[i] > 0.0)) return fail(c, CG_EFOLD, "region %d has non-positive mapped area %g", i, A1[i]);
    res[i] = std::log(A1[i]) - std::log(V[i] * sA1 / sV);
    L += res[i] * res[i];
    sres += res[i];
  }
  double pen = 0.0;
  for (int v = 0; v < nv && !up.custom; ++v) {
    const double dx = X1[v].x - X0[v].x, dy = X1[v].y - X0[v].y;
    pen += dx * dx + dy * dy;
  }
  L += lam * pen;
  if (loss_out && !up.custom) *loss_out = L;
  if (grad_values || grad_blur) {
    std::vector<double> dLdA(R, 0.0), gV(R, 0.0);
    double2* lamX = a->gv;
    double2* lamX2 = a->gv2;
    if (up.custom) {
      // the caller's adjoints: dL/dX' directly, dL/dA' through the shoelace derivative;
      // the loss has no direct dependence on the values here (the caller differentiates
      // any such term itself)
      if (up.g_area) CG_CUDA(c, cudaMemcpy(dLdA.data(), up.g_area, sizeof(double) * R, cudaMemcpyDefault));
      for (int j = 0; j < R; ++j)
        if (!is_finite(dLdA[j])) return fail(c, CG_EINVAL, "area adjoint %d is not finite", j);
      if (up.g_xy) {
        CG_CUDA(c, cudaMemcpyAsync(lamX, up.g_xy, sizeof(double2) * nv, cudaMemcpyDefault, s));
      } else {
        CG_CUDA(c, cudaMemsetAsync(lamX, 0, sizeof(double2) * nv, s));
      }
      CG_CUDA(c, cudaMemcpyAsync(a->dLdA, dLdA.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
      cg::launch_shoelace_adjoint(a->X[K], c->next, c->prev, c->vreg, a->dLdA, lamX, nv, s);
    } else {
      for (int j = 0; j < R; ++j) {
        dLdA[j] = 2.0 * res[j] / A1[j] - 2.0 * sres / sA1;
        gV[j] = -2.0 * res[j] / V[j] + 2.0 * sres / sV;
      }
      CG_CUDA(c, cudaMemcpyAsync(a->dLdA, dLdA.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
      // adjoint of the final vertices
      cg::launch_loss_vertex_adjoint(a->X[K], a->X[0], c->next, c->prev, c->vreg, a->dLdA, lam, lamX, nv, s);
    }
    double dsig_total = 0.0;
    for (int k = K - 1; k >= 0; --k) {
      // the iteration's spectrum, blur factors and integration
      CG_CUDA(c, cudaMemcpyAsync(c->spec64, a->spec[k], sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      cg::launch_blur_tables(nullptr, sigma[k], c->bx, c->by, c->Lx, c->Ly, s);
      // (the replay's buffers are reused by the reverse pass: keep D_k aside; the last
      // iteration's checkpoints and displacements are still those of the forward pass)
      double2* Dk = k == K - 1 ? D_last : adj_replay(c, c->scheds[k], C, true);
      CG_CUDA(c, cudaMemcpyAsync(a->Dk, Dk, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
      // the map X_{k+1} = X_k + D_k(X_k): the displacements' adjoint
      cg::launch_map_adjoint(a->X[k], lamX, (double*)a->lam, c->Lx, c->Ly, nv, s);
      adj_reverse(c, c->scheds[k], C);
      cg::launch_spec_tail(a->lam_spec, c->spec64, c->bx, c->by, sigma[k], a->specp, a->dsig, c->Lx, c->Ly, s);
      cg::launch_inv_rows<double>(c->log2Lx, c->Ly, c->tune.rows, a->specp, a->AB, (const double2*)c->Wx,
                                  (const double2*)c->Ex, c->st, cg::kModeFlux, 0.0, 0, 0, 0u, s);
      cg::launch_inv_cols<double>(c->log2Ly, c->Lx, c->tune.cols, a->AB, a->flux, nullptr, a->dens,
                                  (const double2*)c->Wy, (const double2*)c->Ey, c->st, cg::kModeFlux, s);
      // the iteration's region weights again (for the coverage adjoint of its vertices)
      cg::launch_areas(a->X[k], c->ring_off, c->area_sums, c->reg_off, c->reg_rings, a->vals, R,
                       c->area, c->err_d, c->w, c->info, area_chunks(c), s);
      if (k > 0)
        cg::launch_vertex_map_coverage(a->X[k], c->next, c->vreg, c->w, a->dens, a->Dk, lamX, lamX2, c->Lx, c->Ly,
                                       nv, s);
      cg::launch_raster_adjoint(a->X[k], c->next, c->vreg, a->dens, a->gw, R, c->Lx, c->Ly, nv, s);
      CG_CUDA(c, cudaGetLastError());
      std::vector<double> gw(R);
      double dsig = 0.0;
      CG_CUDA(c, cudaMemcpyAsync(gw.data(), a->gw, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
      CG_CUDA(c, cudaMemcpyAsync(&dsig, a->dsig, sizeof(double), cudaMemcpyDeviceToHost, s));
      CG_CUDA(c, cudaStreamSynchronize(s));
      dsig_total += dsig * decay[k];
      // w_i = (V_i / A_i)(sum A / sum V) - 1
      const std::vector<double>& Ak = A[k];
      double sA = 0.0, sgw = 0.0;
      for (int i = 0; i < R; ++i) sA += Ak[i];
      for (int i = 0; i < R; ++i) sgw += gw[i] * V[i] / Ak[i];
      for (int j = 0; j < R; ++j) gV[j] += gw[j] * sA / (Ak[j] * sV) - sA / (sV * sV) * sgw;
      if (k > 0) {
        // the areas of X_k through the weights
        std::vector<double> dA(R);
        for (int j = 0; j < R; ++j) dA[j] = -gw[j] * V[j] * sA / (Ak[j] * Ak[j] * sV) + sgw / sV;
        CG_CUDA(c, cudaMemcpyAsync(a->dLdA, dA.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
        cg::launch_shoelace_adjoint(a->X[k], c->next, c->prev, c->vreg, a->dLdA, lamX2, nv, s);
        std::swap(lamX, lamX2);
      }
    }
    CG_CUDA(c, cudaGetLastError());
    if (grad_values) CG_CUDA(c, cudaMemcpy(grad_values, gV.data(), sizeof(double) * R, cudaMemcpyDefault));
    if (grad_blur) *grad_blur = dsig_total;
  }
  // leave the context's areas and weights those of its current map and values
  return run_areas(c);
}

template <typename T>
int do_profile(cg_ctx* c, int reps, double* ms_out) {
  cudaStream_t s = c->stream;
  cudaEvent_t a, b;
  CG_CUDA(c, cudaEventCreate(&a));
  CG_CUDA(c, cudaEventCreate(&b));
  const size_t fbytes = sizeof(V2<T>) * (size_t)c->Lx * c->Ly;
  double out[6] = {0, 0, 0, 0, 0, 0};
  CG_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  CG_CUDA(c, cudaMemcpyAsync(c->dbuf[0], c->dres, fbytes, cudaMemcpyDeviceToDevice, s));
  int r0 = ensure_pts(c, c->n_vert);
  if (r0) return r0;
  const double t = 1.0, h = 0.5;
  enqueue_field<T>(c, cg::kModeFixed, t, (V2<T>*)c->vbuf[0], nullptr, nullptr, s);
  enqueue_field<T>(c, cg::kModeFixed, t + h, (V2<T>*)c->vbuf[1], nullptr, nullptr, s);
  cg::launch_gather_u<T>((const V2<T>*)c->vbuf[0], (const V2<T>*)c->dbuf[0], (V2<T>*)c->ubuf[0], c->Lx, c->Ly, s);
  for (int k = 0; k < 6; ++k) {
    CG_CUDA(c, cudaEventRecord(a, s));
    for (int r = 0; r < reps; ++r) {
      switch (k) {
        case 0:
          cg::launch_inv_rows<T>(c->log2Lx, c->Ly, c->tune.rows, (const T*)c->specT, (V2<T>*)c->AB,
                                 (const V2<T>*)c->Wx, (const V2<T>*)c->Ex, c->st, cg::kModeFixed, t + h,
                                 0, 0, 0u, s);
          break;
        case 1:
          launch_cols<T>(c, c->tune.cols, (const V2<T>*)c->AB, (V2<T>*)c->vbuf[1], nullptr, nullptr,
                         cg::kModeFixed, s);
          break;
        case 2:
          cg::launch_heun<T>(c->st, step_params(c), (const V2<T>*)c->vbuf[0], (const V2<T>*)c->vbuf[1],
                             (V2<T>*)c->dbuf[0], (V2<T>*)c->dbuf[1], (V2<T>*)c->ubuf[0], (V2<T>*)c->ubuf[1],
                             c->Lx, c->Ly, cg::kModeFixed, h, 0, 0, c->tune.heun_bps, s);
          break;
        case 3:
          run_raster(c);
          break;
        case 4:
          launch_forward<T>(c, c->bx, c->by, s);  // timing only
          break;
        default:
          cg::launch_map_points<T>(c->xy0, c->pts, c->n_vert, (const V2<T>*)c->dres, c->Lx, c->Ly, s);
          cg::launch_areas(c->xy, c->ring_off, c->area_sums, c->reg_off, c->reg_rings,
                           c->values, c->R_n, c->area, c->err_d, c->w, c->info, area_chunks(c), s);
          break;
      }
    }
    CG_CUDA(c, cudaEventRecord(b, s));
    CG_CUDA(c, cudaEventSynchronize(b));
    float ms = 0.f;
    CG_CUDA(c, cudaEventElapsedTime(&ms, a, b));
    out[k] = ms / reps;
  }
  CG_CUDA(c, cudaGetLastError());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CG_CUDA(c, cudaMemcpy(ms_out, out, sizeof out, cudaMemcpyDefault));
  return CG_OK;
}

void free_adj(cg_ctx* c);

void free_regions(cg_ctx* c) {
  drop_outer_graph(c);  // it holds the map's buffers
  free_adj(c);
  if (c->prev) cudaFree(c->prev);
  c->prev = nullptr;
  c->scheds.clear();
  void* ps[] = {c->values, c->ring_off, c->reg_off, c->reg_rings, c->next, c->vreg,
                c->xy, c->xy0, c->area_sums, c->area, c->err_d, c->w, c->chunk_ring, c->ring_chunk_off,
                c->chunk_sum};
  for (void* p : ps)
    if (p) cudaFree(p);
  c->chunk_ring = nullptr; c->ring_chunk_off = nullptr; c->chunk_sum = nullptr; c->n_chunks = 0;
  c->values = nullptr; c->ring_off = nullptr; c->reg_off = nullptr; c->reg_rings = nullptr;
  c->next = nullptr; c->vreg = nullptr; c->xy = nullptr; c->xy0 = nullptr;
  c->area_sums = nullptr; c->area = nullptr; c->err_d = nullptr; c->w = nullptr;
  c->map_off.clear();
  c->map_reg.clear();
  c->have_regions = false;
}

// ---- batches -------------------------------------------------------------------

int batch_fail(cg_batch* b, int code, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  b->err = buf;
  return code;
}

// One graph, one branch per context: fork from a common node, each branch the
// context's whole outer iteration (capture_cartogram), join at the end.
int batch_build(cg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  const size_t n = b->ctx.size();
  std::vector<cudaStream_t> br(n, nullptr);
  cudaStream_t ms = nullptr, bs = nullptr, bs2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(ms, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      e = cudaEventRecord(fork, ms);
      for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cg_ctx* c = b->ctx[i];
        e = cudaStreamWaitEvent(br[i], fork, 0);
        if (e == cudaSuccess)
          e = c->mixed ? capture_cartogram<float>(c, br[i], bs, bs2) : capture_cartogram<double>(c, br[i], bs, bs2);
        if (e == cudaSuccess) e = cudaEventRecord(join, br[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ms, join, 0);
      }
      const cudaError_t e2 = cudaStreamEndCapture(ms, &g);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  int rc = CG_OK;
  if (e == cudaSuccess) {
    b->graph = g;
    for (size_t i = 0; i < n; ++i) b->gen[i] = b->ctx[i]->gen;
  } else {
    rc = batch_fail(b, CG_ECUDA, "batch graph capture", e);
    if (g) cudaGraphDestroy(g);
    b->exec = nullptr;
  }
  cudaGetLastError();
  for (cudaStream_t st : br)
    if (st) cudaStreamDestroy(st);
  if (ms) cudaStreamDestroy(ms);
  if (bs) cudaStreamDestroy(bs);
  if (bs2) cudaStreamDestroy(bs2);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  return rc;
}

template <typename T>
int batch_begin(cg_ctx* c, cg_stats& s, bool* go) {
  int r = maybe_tune_first<T>(c, s, go);
  if (r || !*go) return r;
  return outer_prepare<T>(c, c->opt.max_iter - s.iterations);
}

}  // namespace

// ============================================================================
// C-ABI
// ============================================================================

extern "C" {

int cartogram_default_options(cg_options* o) {
  if (!o) return CG_EINVAL;
  o->precision = CG_PRECISION_FP64;
  o->dt0 = 1e-2;
  o->atol = 1e-2;
  o->grow = 1.2;
  o->shrink = 0.5;
  o->cfl = 1.0;
  o->rho_tol = 1e-4;
  o->area_tol = 0.01;
  o->max_steps = 4000;
  o->max_iter = 500;
  o->use_graph = 1;
  o->blur_decay = 0.5;
  o->autotune = 1;
  o->flow = CG_FLOW_DIFFUSION;
  o->time_limit = 0.0;
  o->barrier_spins = 1ll << 25;
  return CG_OK;
}

int cartogram_init(int Lx, int Ly, double blur_width, const cg_options* opt, cg_ctx** out) {
  if (!out) return CG_EINVAL;
  *out = nullptr;
  if (!pow2_in_range(Lx) || !pow2_in_range(Ly)) return CG_EINVAL;
  if (!is_finite(blur_width) || blur_width < 0.0) return CG_EINVAL;
  cg_options o;
  cartogram_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != CG_PRECISION_FP64 && o.precision != CG_PRECISION_MIXED && o.precision != CG_PRECISION_MIXED_FF)
    return CG_EINVAL;
  if (o.use_graph < 0 || o.use_graph > 2) return CG_EINVAL;
  if (o.flow != CG_FLOW_DIFFUSION && o.flow != CG_FLOW_LINEAR) return CG_EINVAL;
  if (!is_finite(o.time_limit) || o.time_limit < 0.0 || o.time_limit > 1e9) return CG_EINVAL;
  if (o.barrier_spins < 1 || o.barrier_spins > (1ll << 40)) return CG_EINVAL;
  if (!(o.dt0 > 0) || !(o.atol > 0) || !(o.grow >= 1.0) || !(o.shrink > 0 && o.shrink < 1) ||
      !(o.cfl > 0) || !(o.rho_tol > 0) || !(o.area_tol > 0) || o.max_steps < 1 || o.max_iter < 0 ||
      !is_finite(o.dt0) || !is_finite(o.atol) || !is_finite(o.grow) || !is_finite(o.cfl) || !is_finite(o.rho_tol) ||
      !is_finite(o.area_tol))
    return CG_EINVAL;
  cg_ctx* c = new cg_ctx();
  c->Lx = Lx;
  c->Ly = Ly;
  c->log2Lx = ilog2(Lx);
  c->log2Ly = ilog2(Ly);
  c->blur = blur_width;
  c->opt = o;
  c->mixed = o.precision != CG_PRECISION_FP64;
  c->ff = o.precision == CG_PRECISION_MIXED_FF;
  int r = CG_OK;
  if (cudaGetDevice(&c->device) != cudaSuccess) r = CG_ECUDA;
  if (!r && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) r = CG_ECUDA;
  c->stream = c->own_stream;
  if (!r && (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)) r = CG_ECUDA;
  if (!r) r = c->mixed ? alloc_fields<float>(c) : alloc_fields<double>(c);
  if (r) {
    cudaGetLastError();
    cartogram_destroy(c);
    return r;
  }
  *out = c;
  return CG_OK;
}

int cartogram_set_stream(cg_ctx* c, void* stream) {
  int r = check_ctx(c, false);
  if (r) return r;
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return CG_OK;
}

// The areas of a newly set map; every region needs a positive one (else the map is dropped).
int check_areas(cg_ctx* c) {
  int r;
  if ((r = run_areas(c)) || (r = read_info(c))) return r;
  std::vector<double> area(c->R_n);
  CG_CUDA(c, cudaMemcpy(area.data(), c->area, sizeof(double) * c->R_n, cudaMemcpyDeviceToHost));
  for (int k = 0; k < c->R_n; ++k)
    if (!(area[k] > 0.0)) {
      free_regions(c);
      return fail(c, CG_EINVAL, "region %d has non-positive area %g", k, area[k]);
    }
  return CG_OK;
}

int cartogram_set_regions(cg_ctx* c, int n_regions, const double* target_values, int64_t n_rings,
                          const int64_t* ring_offsets, const int32_t* ring_region,
                          const double* xy) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (n_regions < 1 || n_rings < 1 || !target_values || !ring_offsets || !ring_region || !xy)
    return fail(c, CG_EINVAL, "empty map or NULL array");
  if (n_rings > (1LL << 30)) return fail(c, CG_EINVAL, "too many rings");
  // inputs may live on the host or the device: bring them to the host to validate
  std::vector<double> vals(n_regions);
  std::vector<long long> off(n_rings + 1);
  std::vector<int> reg(n_rings);
  CG_CUDA(c, cudaMemcpy(vals.data(), target_values, sizeof(double) * n_regions, cudaMemcpyDefault));
  CG_CUDA(c, cudaMemcpy(off.data(), ring_offsets, sizeof(long long) * (n_rings + 1), cudaMemcpyDefault));
  CG_CUDA(c, cudaMemcpy(reg.data(), ring_region, sizeof(int) * n_rings, cudaMemcpyDefault));
  for (int k = 0; k < n_regions; ++k)
    if (!is_finite(vals[k]) || !(vals[k] > 0.0)) return fail(c, CG_EINVAL, "target value %d is not positive and finite", k);
  if (off[0] != 0) return fail(c, CG_EINVAL, "ring_offsets[0] must be 0");
  for (long long k = 0; k < n_rings; ++k) {
    if (off[k + 1] - off[k] < 3) return fail(c, CG_EINVAL, "ring %lld has fewer than 3 vertices", k);
    if (reg[k] < 0 || reg[k] >= n_regions) return fail(c, CG_EINVAL, "ring %lld has region %d out of range", k, reg[k]);
  }
  const long long nv = off[n_rings];
  if (nv >= (1LL << 31)) return fail(c, CG_EINVAL, "too many vertices");
  // the vertices are validated where they are when that is host memory, else from a copy
  std::vector<double> pts;
  const double* hxy = xy;
  {
    cudaPointerAttributes pa;
    const bool dev = cudaPointerGetAttributes(&pa, xy) == cudaSuccess &&
                     (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
      pts.resize(2 * (size_t)nv);
      CG_CUDA(c, cudaMemcpy(pts.data(), xy, sizeof(double) * 2 * nv, cudaMemcpyDefault));
      hxy = pts.data();
    }
  }
  for (long long k = 0; k < nv; ++k) {
    const double x = hxy[2 * k], y = hxy[2 * k + 1];
    if (!is_finite(x) || !is_finite(y) || x < 0.0 || x > c->Lx || y < 0.0 || y > c->Ly)
      return fail(c, CG_EINVAL, "vertex %lld (%g, %g) is outside the box [0,%d]x[0,%d]", k, x, y, c->Lx, c->Ly);
  }
  if (c->have_regions && n_regions == c->R_n && off == c->map_off && reg == c->map_reg) {
    // the same rings: keep every buffer (and the graphs and work spaces that hold them)
    c->scheds.clear();
    CG_CUDA(c, cudaMemcpy(c->values, vals.data(), sizeof(double) * n_regions, cudaMemcpyHostToDevice));
    CG_CUDA(c, cudaMemcpy(c->xy, xy, sizeof(double2) * nv, cudaMemcpyDefault));
    CG_CUDA(c, cudaMemcpy(c->xy0, c->xy, sizeof(double2) * nv, cudaMemcpyDeviceToDevice));
    c->hist_len = 0;
    c->have_spectrum = false;
    return check_areas(c);
  }
  // per-vertex successor and region, region -> rings index
  std::vector<int> next(nv), vreg(nv), reg_off(n_regions + 1, 0), reg_rings(n_rings);
  for (long long k = 0; k < n_rings; ++k) {
    for (long long v = off[k]; v < off[k + 1]; ++v) {
      next[v] = (int)(v + 1 < off[k + 1] ? v + 1 : off[k]);
      vreg[v] = reg[k];
    }
    reg_off[reg[k] + 1]++;
  }
  for (int k = 0; k < n_regions; ++k) reg_off[k + 1] += reg_off[k];
  {
    std::vector<int> fill(reg_off.begin(), reg_off.end() - 1);
    for (long long k = 0; k < n_rings; ++k) reg_rings[fill[reg[k]]++] = (int)k;
  }
  free_regions(c);
  c->R_n = n_regions;
  c->n_rings = n_rings;
  c->n_vert = nv;
  CG_CUDA(c, cudaMalloc((void**)&c->values, sizeof(double) * n_regions));
  CG_CUDA(c, cudaMalloc((void**)&c->ring_off, sizeof(long long) * (n_rings + 1)));
  CG_CUDA(c, cudaMalloc((void**)&c->reg_off, sizeof(int) * (n_regions + 1)));
  CG_CUDA(c, cudaMalloc((void**)&c->reg_rings, sizeof(int) * n_rings));
  CG_CUDA(c, cudaMalloc((void**)&c->next, sizeof(int) * nv));
  CG_CUDA(c, cudaMalloc((void**)&c->vreg, sizeof(int) * nv));
  CG_CUDA(c, cudaMalloc((void**)&c->xy, sizeof(double2) * nv));
  CG_CUDA(c, cudaMalloc((void**)&c->xy0, sizeof(double2) * nv));
  CG_CUDA(c, cudaMalloc((void**)&c->area_sums, sizeof(double) * 2));
  CG_CUDA(c, cudaMalloc((void**)&c->area, sizeof(double) * n_regions));
  CG_CUDA(c, cudaMalloc((void**)&c->err_d, sizeof(double) * n_regions));
  CG_CUDA(c, cudaMalloc((void**)&c->w, sizeof(double) * n_regions));
  CG_CUDA(c, cudaMemcpy(c->values, vals.data(), sizeof(double) * n_regions, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(c->ring_off, off.data(), sizeof(long long) * (n_rings + 1), cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(c->reg_off, reg_off.data(), sizeof(int) * (n_regions + 1), cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(c->reg_rings, reg_rings.data(), sizeof(int) * n_rings, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(c->next, next.data(), sizeof(int) * nv, cudaMemcpyHostToDevice));
  CG_CUDA(c, cudaMemcpy(c->vreg, vreg.data(), sizeof(int) * nv, cudaMemcpyHostToDevice));
  {
    // the area sums' chunks: up to kAreaChunk consecutive vertices of one ring
    std::vector<int> ring_chunk_off(n_rings + 1, 0), chunk_ring;
    for (long long k = 0; k < n_rings; ++k) {
      const long long nk = (off[k + 1] - off[k] + cg::kAreaChunk - 1) / cg::kAreaChunk;
      ring_chunk_off[k + 1] = ring_chunk_off[k] + (int)nk;
      for (long long q = 0; q < nk; ++q) chunk_ring.push_back((int)k);
    }
    c->n_chunks = (long long)chunk_ring.size();
    CG_CUDA(c, cudaMalloc((void**)&c->ring_chunk_off, sizeof(int) * (n_rings + 1)));
    CG_CUDA(c, cudaMalloc((void**)&c->chunk_ring, sizeof(int) * std::max<long long>(1, c->n_chunks)));
    CG_CUDA(c, cudaMalloc((void**)&c->chunk_sum, sizeof(double) * std::max<long long>(1, c->n_chunks)));
    CG_CUDA(c, cudaMemcpy(c->ring_chunk_off, ring_chunk_off.data(), sizeof(int) * (n_rings + 1),
                          cudaMemcpyHostToDevice));
    if (c->n_chunks > 0)
      CG_CUDA(c, cudaMemcpy(c->chunk_ring, chunk_ring.data(), sizeof(int) * c->n_chunks, cudaMemcpyHostToDevice));
  }
  {
    std::vector<int> prev(nv);
    for (long long v = 0; v < nv; ++v) prev[next[v]] = (int)v;
    CG_CUDA(c, cudaMalloc((void**)&c->prev, sizeof(int) * nv));
    CG_CUDA(c, cudaMemcpy(c->prev, prev.data(), sizeof(int) * nv, cudaMemcpyHostToDevice));
  }
  CG_CUDA(c, cudaMemcpy(c->xy, xy, sizeof(double2) * nv, cudaMemcpyDefault));
  CG_CUDA(c, cudaMemcpy(c->xy0, c->xy, sizeof(double2) * nv, cudaMemcpyDeviceToDevice));
  c->have_regions = true;
  c->hist_len = 0;
  c->have_spectrum = false;
  c->map_off = std::move(off);
  c->map_reg = std::move(reg);
  return check_areas(c);
}

int cartogram_integrate(cg_ctx* c, cg_stats* stats) {
  int r = check_ctx(c, true);
  if (r) return r;
  return c->mixed ? do_integrate<float>(c, stats) : do_integrate<double>(c, stats);
}

int cartogram_project(cg_ctx* c, int64_t n, const double* xy_in, double* xy_out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (n < 0 || (n > 0 && (!xy_in || !xy_out))) return fail(c, CG_EINVAL, "bad point array");
  return c->mixed ? do_project<float>(c, n, xy_in, xy_out) : do_project<double>(c, n, xy_in, xy_out);
}

int cartogram_area_errors(cg_ctx* c, double* err) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!err) return fail(c, CG_EINVAL, "NULL output");
  if ((r = run_areas(c)) || (r = read_info(c))) return r;
  CG_CUDA(c, cudaMemcpy(err, c->err_d, sizeof(double) * c->R_n, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_get_vertices(cg_ctx* c, double* xy_out) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!xy_out) return fail(c, CG_EINVAL, "NULL output");
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  CG_CUDA(c, cudaMemcpy(xy_out, c->xy, sizeof(double2) * c->n_vert, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_reset(cg_ctx* c) {
  int r = check_ctx(c, true);
  if (r) return r;
  CG_CUDA(c, cudaMemcpyAsync(c->xy, c->xy0, sizeof(double2) * c->n_vert, cudaMemcpyDeviceToDevice, c->stream));
  c->hist_len = 0;
  return CG_OK;
}

int cartogram_polygon_measures(cg_ctx* c, double* out) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!out) return fail(c, CG_EINVAL, "NULL output");
  const int R = c->R_n, nb = cg::polygon_blocks(R);
  double* scratch = nullptr;  // cent [2R][2], alpha [R], part [nb], result [3]
  CG_CUDA(c, cudaMalloc((void**)&scratch, sizeof(double) * (5 * (size_t)R + nb + 3)));
  double2* cent = (double2*)scratch;
  double* alpha = scratch + 4 * (size_t)R;
  double* part = alpha + R;
  double* res = part + nb;
  cg::launch_polygon_measures(c->xy, c->xy0, c->ring_off, c->reg_off, c->reg_rings, R, cent, alpha, part, res,
                              c->stream);
  double h[3];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(scratch);
  if (e != cudaSuccess) return fail(c, CG_ECUDA, "polygon measures: %s", cudaGetErrorString(e));
  CG_CUDA(c, cudaMemcpy(out, h, sizeof h, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_set_values(cg_ctx* c, const double* target_values) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!target_values) return fail(c, CG_EINVAL, "NULL values");
  std::vector<double> vals(c->R_n);
  CG_CUDA(c, cudaMemcpy(vals.data(), target_values, sizeof(double) * c->R_n, cudaMemcpyDefault));
  for (int k = 0; k < c->R_n; ++k)
    if (!is_finite(vals[k]) || !(vals[k] > 0.0)) return fail(c, CG_EINVAL, "target value %d is not positive and finite", k);
  CG_CUDA(c, cudaMemcpyAsync(c->values, vals.data(), sizeof(double) * c->R_n, cudaMemcpyHostToDevice, c->stream));
  CG_CUDA(c, cudaMemcpyAsync(c->xy, c->xy0, sizeof(double2) * c->n_vert, cudaMemcpyDeviceToDevice, c->stream));
  c->hist_len = 0;
  c->have_spectrum = false;
  c->scheds.clear();
  if ((r = run_areas(c))) return r;
  CG_CUDA(c, cudaStreamSynchronize(c->stream));  // vals is released on return
  return CG_OK;
}

int cartogram_profile(cg_ctx* c, int reps, double* ms_out) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!c->have_spectrum) return fail(c, CG_ESTATE, "no spectrum: run an integration first");
  if (reps < 1 || !ms_out) return fail(c, CG_EINVAL, "bad profile arguments");
  return c->mixed ? do_profile<float>(c, reps, ms_out) : do_profile<double>(c, reps, ms_out);
}

int cartogram_read_bandwidth(int64_t bytes, int passes, double* gbs_out) {
  if (bytes < (1 << 20) || bytes > (int64_t)64 << 30 || (bytes & 15) || passes < 1 || passes > 1000 || !gbs_out)
    return CG_EINVAL;
  void* buf = nullptr;
  float* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = CG_OK;
  if (cudaMalloc(&buf, (size_t)bytes) != cudaSuccess || cudaMalloc((void**)&sink, 64) != cudaSuccess) rc = CG_ENOMEM;
  if (!rc && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    rc = CG_ECUDA;
  if (!rc && cudaMemsetAsync(buf, 0, (size_t)bytes, s) != cudaSuccess) rc = CG_ECUDA;
  float best = 1e30f;
  for (int round = 0; round < 4 && !rc; ++round) {
    cg::launch_read_bw(buf, (size_t)bytes, 1, sink, s);  // brings a buffer that fits in L2 there
    cudaEventRecord(a, s);
    cg::launch_read_bw(buf, (size_t)bytes, passes, sink, s);
    cudaEventRecord(b, s);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) rc = CG_ECUDA;
    else if (round > 0) best = std::min(best, ms);  // round 0 warms up
  }
  if (!rc) *gbs_out = (double)bytes * passes / (best * 1e-3) / 1e9;
  if (b) cudaEventDestroy(b);
  if (a) cudaEventDestroy(a);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (buf) cudaFree(buf);
  cudaGetLastError();
  return rc;
}

int cartogram_autotune(cg_ctx* c, int reps, int* shapes_out, double* ms_out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (reps < 0) return fail(c, CG_EINVAL, "reps must not be negative");
  if (reps > 0) {
    r = c->mixed ? do_autotune<float>(c, reps) : do_autotune<double>(c, reps);
    if (r) return r;
  }
  const int shp[3] = {c->tune.rows, c->tune.cols, c->tune.heun_bps};
  if (shapes_out) CG_CUDA(c, cudaMemcpy(shapes_out, shp, sizeof shp, cudaMemcpyDefault));
  if (ms_out) CG_CUDA(c, cudaMemcpy(ms_out, c->tune_ms, sizeof c->tune_ms, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_fold_count(cg_ctx* c, int k, long long* n_folded, double* min_area) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (k < 0 || k >= c->hist_len) return fail(c, CG_EINVAL, "history entry %d out of range", k);
  unsigned long long* d = (unsigned long long*)c->acc2;  // scratch: the persistent kernel's slots
  if (c->mixed) cg::launch_fold_count<float>((const V2<float>*)c->hist[k], c->Lx, c->Ly, d, c->stream);
  else cg::launch_fold_count<double>((const V2<double>*)c->hist[k], c->Lx, c->Ly, d, c->stream);
  CG_CUDA(c, cudaGetLastError());
  unsigned long long h[2];
  CG_CUDA(c, cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  const unsigned long long b = (h[1] & 0x8000000000000000ull) ? (h[1] & 0x7fffffffffffffffull) : ~h[1];
  double mn;
  memcpy(&mn, &b, sizeof mn);
  if (n_folded) *n_folded = (long long)h[0];
  if (min_area) *min_area = mn;
  return CG_OK;
}

int cartogram_history_length(const cg_ctx* c) { return c ? c->hist_len : 0; }

int cartogram_iteration_record(cg_ctx* c, int k, double* out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (k < 0 || k >= c->hist_len || !out) return fail(c, CG_EINVAL, "history entry %d out of range", k);
  const size_t fbytes = (c->mixed ? sizeof(float2) : sizeof(double2)) * (size_t)c->Lx * c->Ly;
  cg::IterRecord rec;
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  CG_CUDA(c, cudaMemcpy(&rec, static_cast<const char*>(c->hist[k]) + fbytes, sizeof rec, cudaMemcpyDeviceToHost));
  const double o[6] = {rec.max_err, rec.t_end, (double)rec.accepted, (double)rec.rejected, rec.loop_ns * 1e-6,
                       rec.blur};
  CG_CUDA(c, cudaMemcpy(out, o, sizeof o, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_get_grid(cg_ctx* c, int k, double* xy_out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (k < 0 || k >= c->hist_len || !xy_out) return fail(c, CG_EINVAL, "history entry %d out of range", k);
  return c->mixed ? grid_out<float>(c, c->hist[k], xy_out) : grid_out<double>(c, c->hist[k], xy_out);
}

int cartogram_density(cg_ctx* c, double* rho_out) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (!rho_out) return fail(c, CG_EINVAL, "NULL output");
  if ((r = run_areas(c)) || (r = run_raster(c))) return r;
  const size_t N = (size_t)c->Lx * c->Ly;
  std::vector<double> h(N);
  CG_CUDA(c, cudaMemcpyAsync(h.data(), c->acc, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  for (double& v : h) v += 1.0;
  CG_CUDA(c, cudaMemcpy(rho_out, h.data(), sizeof(double) * N, cudaMemcpyDefault));
  return CG_OK;
}

int cartogram_spectrum(cg_ctx* c, double* spec_out) {
  int r = check_ctx(c, true);
  if (r) return r;
  if ((r = run_areas(c)) || (r = run_raster(c))) return r;
  r = c->mixed ? run_forward<float>(c) : run_forward<double>(c);
  if (r) return r;
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (spec_out) {
    const size_t N = (size_t)c->Lx * c->Ly;
    std::vector<double> h(N);
    CG_CUDA(c, cudaMemcpy(h.data(), c->spec64, sizeof(double) * N, cudaMemcpyDeviceToHost));
    h[0] = (double)c->Lx * c->Ly;
    CG_CUDA(c, cudaMemcpy(spec_out, h.data(), sizeof(double) * N, cudaMemcpyDefault));
  }
  return CG_OK;
}

int cartogram_velocity(cg_ctx* c, double t, double* rho_out, double* v_out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (!c->have_spectrum) return fail(c, CG_ESTATE, "no spectrum: call cartogram_spectrum first");
  if (!is_finite(t) || t < 0.0) return fail(c, CG_EINVAL, "bad time %g", t);
  return c->mixed ? do_velocity<float>(c, t, rho_out, v_out) : do_velocity<double>(c, t, rho_out, v_out);
}

int cartogram_heun_step(cg_ctx* c, double t, double h, const double* disp_in, double* disp_out,
                        double* err) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (!c->have_spectrum) return fail(c, CG_ESTATE, "no spectrum: call cartogram_spectrum first");
  if (!is_finite(t) || t < 0.0 || !is_finite(h) || !(h > 0.0) || !disp_in || !disp_out)
    return fail(c, CG_EINVAL, "bad step arguments");
  return c->mixed ? do_heun<float>(c, t, h, disp_in, disp_out, err)
                  : do_heun<double>(c, t, h, disp_in, disp_out, err);
}

int cartogram_integrate_once(cg_ctx* c, double* grid_out, long long* accepted, long long* rejected,
                             double* t_end) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (!c->have_spectrum) return fail(c, CG_ESTATE, "no spectrum: call cartogram_spectrum first");
  return c->mixed ? do_integrate_once<float>(c, grid_out, accepted, rejected, t_end)
                  : do_integrate_once<double>(c, grid_out, accepted, rejected, t_end);
}

int cartogram_distortion(cg_ctx* c, double* out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (!out) return fail(c, CG_EINVAL, "NULL output");
  return c->mixed ? do_distortion<float>(c, out) : do_distortion<double>(c, out);
}

int cartogram_inverse_project(cg_ctx* c, int64_t n, const double* xy_in, double* xy_out) {
  int r = check_ctx(c, false);
  if (r) return r;
  if (n < 0 || (n > 0 && (!xy_in || !xy_out))) return fail(c, CG_EINVAL, "bad point array");
  return c->mixed ? do_inverse_project<float>(c, n, xy_in, xy_out) : do_inverse_project<double>(c, n, xy_in, xy_out);
}

int cartogram_iteration_gradient(cg_ctx* c, const double* values, double blur_width, double lambda, int iterations,
                                 int replay, int checkpoint, double* loss, double* grad_values, double* grad_blur) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (c->mixed || c->opt.flow != CG_FLOW_DIFFUSION)
    return fail(c, CG_EINVAL, "the gradient needs the FP64 path and the diffusion flow");
  if (!values || !is_finite(blur_width) || blur_width < 0.0 || !is_finite(lambda) || lambda < 0.0 || checkpoint < 1 ||
      iterations < 1)
    return fail(c, CG_EINVAL, "bad gradient arguments");
  if (!loss && !grad_values && !grad_blur) return fail(c, CG_EINVAL, "no output");
  return do_iteration_gradient(c, values, blur_width, lambda, iterations, replay, checkpoint, loss, grad_values,
                               grad_blur);
}

int cartogram_iteration_vjp(cg_ctx* c, const double* values, double blur_width, int iterations, int replay,
                            int checkpoint, double* xy_out, double* area_out, const double* grad_xy,
                            const double* grad_area, double* grad_values, double* grad_blur) {
  int r = check_ctx(c, true);
  if (r) return r;
  if (c->mixed || c->opt.flow != CG_FLOW_DIFFUSION)
    return fail(c, CG_EINVAL, "the gradient needs the FP64 path and the diffusion flow");
  if (!values || !is_finite(blur_width) || blur_width < 0.0 || checkpoint < 1 || iterations < 1)
    return fail(c, CG_EINVAL, "bad gradient arguments");
  if (!xy_out && !area_out && !grad_values && !grad_blur) return fail(c, CG_EINVAL, "no output");
  Upstream up;
  up.custom = true;
  up.g_xy = grad_xy;
  up.g_area = grad_area;
  up.xy_out = xy_out;
  up.area_out = area_out;
  return do_iteration_gradient(c, values, blur_width, 0.0, iterations, replay, checkpoint, nullptr, grad_values,
                               grad_blur, up);
}

const char* cartogram_last_error(const cg_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void cartogram_destroy(cg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  free_regions(c);
  void* ps[] = {c->Wx, c->Wy, c->Ex, c->Ey, c->Wyff, c->Eyff, c->Wfxff, c->Efxff, c->Wfyff, c->Efyff, c->Wfx, c->Wfy, c->Efx, c->Efy, c->bx, c->by,
                c->acc, c->R, c->spec64, c->AB, c->vbuf[0], c->vbuf[1], c->dbuf[0], c->dbuf[1],
                c->ubuf[0], c->ubuf[1], c->dres, c->rho_tmp, c->st, c->info, c->pts, c->gb, c->acc2, c->phi, c->flux,
                c->rho0, c->diag, c->deadline};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (c->specT && c->specT != c->spec64) cudaFree(c->specT);
  for (void* p : c->hist) cudaFree(p);
  if (c->info_h) cudaFreeHost(c->info_h);
  free_adj(c);
  if (c->outer) cudaFree(c->outer);
  if (c->outer_h) cudaFreeHost(c->outer_h);
  if (c->sigma_d) cudaFree(c->sigma_d);
  if (c->sigma_h) cudaFreeHost(c->sigma_h);
  if (c->hist_d) cudaFree(c->hist_d);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  cudaGetLastError();
  delete c;
}

int cartogram_batch_create(cg_ctx* const* ctxs, int n, cg_batch** out) {
  if (!out) return CG_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) return CG_EINVAL;
  std::vector<cg_ctx*> v(ctxs, ctxs + n);
  for (int i = 0; i < n; ++i) {
    if (!v[i]) return CG_EINVAL;
    for (int k = 0; k < i; ++k)
      if (v[k] == v[i]) return CG_EINVAL;
    if (v[i]->device != v[0]->device) return CG_EINVAL;
  }
  cg_batch* b = new cg_batch();
  b->ctx = v;
  b->gen.assign(n, 0);
  b->device = v[0]->device;
  if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return CG_ECUDA;
  }
  *out = b;
  return CG_OK;
}

int cartogram_batch_integrate(cg_batch* b, cg_stats* stats, int* status) {
  if (!b) return CG_EINVAL;
  b->err.clear();
  if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, CG_ECUDA, "cudaSetDevice", cudaGetLastError());
  const auto t0 = std::chrono::steady_clock::now();
  const size_t n = b->ctx.size();
  std::vector<cg_stats> st(n);
  std::vector<int> rc(n, CG_OK);
  std::vector<char> go(n, 0);
  for (size_t i = 0; i < n; ++i) {
    cg_ctx* c = b->ctx[i];
    memset(&st[i], 0, sizeof(cg_stats));
    c->err.clear();
    if (!c->have_regions) {
      rc[i] = fail(c, CG_ESTATE, "no map: call cartogram_set_regions first");
      continue;
    }
    stamp_deadline(c);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      rc[i] = fail(c, CG_ECUDA, "stream synchronisation failed");
      continue;
    }
    bool g = false;
    rc[i] = c->mixed ? batch_begin<float>(c, st[i], &g) : batch_begin<double>(c, st[i], &g);
    go[i] = rc[i] == CG_OK && g;
  }
  bool any = false;
  for (size_t i = 0; i < n; ++i) any |= go[i] != 0;
  if (any) {
    // branches of contexts that are done (or failed) skip their loop
    for (size_t i = 0; i < n; ++i) {
      if (go[i]) continue;
      cg_ctx* c = b->ctx[i];
      if (!c->have_regions) continue;
      cg::OuterState o;
      memset(&o, 0, sizeof o);
      o.status = cg::kOuterConverged;
      o.max_iter = 0;
      if (cudaMemcpy(c->outer, &o, sizeof o, cudaMemcpyHostToDevice) != cudaSuccess)
        return batch_fail(b, CG_ECUDA, "batch state", cudaGetLastError());
    }
    bool stale = !b->exec;
    for (size_t i = 0; i < n; ++i) stale |= b->gen[i] != b->ctx[i]->gen || !b->ctx[i]->have_regions;
    if (stale) {
      for (size_t i = 0; i < n; ++i)
        if (!b->ctx[i]->have_regions) return batch_fail(b, CG_ESTATE, "a context has no map", cudaSuccess);
      int r = batch_build(b);
      if (r) return r;
    }
    for (;;) {
      cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
      for (size_t i = 0; i < n && e == cudaSuccess; ++i)
        if (go[i])
          e = cudaMemcpyAsync(b->ctx[i]->outer_h, b->ctx[i]->outer, sizeof(cg::OuterState), cudaMemcpyDeviceToHost,
                              b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return batch_fail(b, CG_ECUDA, "batch launch", e);
      bool again = false;
      for (size_t i = 0; i < n; ++i) {
        if (!go[i] || b->ctx[i]->outer_h->status != cg::kOuterNeedSlots) continue;
        cg_ctx* c = b->ctx[i];
        const int r = c->mixed ? outer_resume<float>(c) : outer_resume<double>(c);
        if (r) {
          rc[i] = r;
          go[i] = 0;
          cg::OuterState o;
          memset(&o, 0, sizeof o);
          o.status = cg::kOuterConverged;
          cudaMemcpy(c->outer, &o, sizeof o, cudaMemcpyHostToDevice);
          continue;
        }
        again = true;
      }
      if (!again) break;
    }
    for (size_t i = 0; i < n; ++i)
      if (go[i]) rc[i] = outer_finish(b->ctx[i], st[i]);
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int first = CG_OK;
  for (size_t i = 0; i < n; ++i) {
    st[i].converged = st[i].max_area_error < b->ctx[i]->opt.area_tol;
    st[i].seconds = secs;
    if (stats) stats[i] = st[i];
    if (status) status[i] = rc[i];
    if (first == CG_OK && rc[i] != CG_OK) {
      first = rc[i];
      b->err = "context " + std::to_string(i) + ": " + b->ctx[i]->err;
    }
  }
  return first;
}

const char* cartogram_batch_last_error(const cg_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

void cartogram_batch_destroy(cg_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
