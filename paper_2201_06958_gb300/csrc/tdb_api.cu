// tdb_api.cu - the C ABI of libtdb: context, workspace layout, the step driver,
// HOSVD (re)initialisation and the add/remove-mode rule of Sec. 2.5.
//
// Step (Secs. 2.2, 2.3): dV = V_{k+1} - V_k; dS and Y_n by the projection of
// Eqs. 2.15/2.16; X_n = Y_(n) T_(n)^T (T_(n) T_(n)^T)^{-1}; dU_n = (I - U U^T W) X_n;
// T += dS, U_n += dU_n (explicit Euler, dt cancels); weighted Cholesky-QR with core
// compensation; error (Eq. 2.20) when scheduled; rank control (Sec. 2.5).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "mlp.h"
#include "tc_project.h"

namespace tdb {

static thread_local std::string g_init_error;


enum Action { ACT_NONE = 0, ACT_REINIT = 1, ACT_INCREASE = 2, ACT_DECREASE = 3, ACT_REVERT = 4, ACT_CAP = 5 };

struct Readback {
  double err2;
  double dv2;
  double ds2;
  double est;                      // estimator output (error, not log)
  double sig2[kMaxModes][kMaxRank];
  float feat[MLP_F];               // estimator features of this step
  int need;                        // 1: the exact error was evaluated this step
  unsigned flags;
};

// The step's first kernel: clears the step record, fetches the host's gate word and the
// estimator state from pinned host memory (read through its device mapping), keeps the
// sigma^2 the step starts from (the estimator's features), and lets the projection that
// follows start its set-up early (programmatic launch).  One CTA.
__global__ void k_step_begin(Readback* rb, const int* need_h, const EstState* est_h, EstState* est_d,
                             const double* sig2, double* sig2_lag, int nsig) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  unsigned* w = (unsigned*)rb;
  for (int i = threadIdx.x; i < (int)(sizeof(Readback) / 4); i += blockDim.x) w[i] = 0u;
  const unsigned* es = (const unsigned*)est_h;
  unsigned* ed = (unsigned*)est_d;
  for (int i = threadIdx.x; i < (int)(sizeof(EstState) / 4); i += blockDim.x) ed[i] = es[i];
  for (int i = threadIdx.x; i < nsig; i += blockDim.x) sig2_lag[i] = sig2[i];
  __syncthreads();
  if (threadIdx.x == 0) rb->need = *(volatile const int*)need_h;
}

}  // namespace tdb

using namespace tdb;

struct tdb_ctx {
  tdb_config cfg;
  int p = 0;
  int64_t N[kMaxModes] = {0};
  int64_t S = 0;
  int r[kMaxModes] = {0};
  int cap[kMaxModes] = {0};
  int kcap[kMaxModes] = {0};      // eigenpairs kept from each HOSVD
  int prec = 0;
  bool f64 = false;
  size_t esz = 4;                 // snapshot element size
  cudaStream_t stream = nullptr;
  std::string err;

  // device buffers
  double* w[kMaxModes];
  double* U[kMaxModes];
  double* Up[kMaxModes];
  double* X[kMaxModes];
  void* A[kMaxModes];
  void* Uc[kMaxModes];
  double* Ubak[kMaxModes];
  double* T;
  double* T2;
  double* Tbak;
  void* Tcore;                    // compute-type core (alias of T in FP64 mode)
  void* dS;
  void* Y[kMaxModes];
  void* dV;
  void* ping;
  void* pong;
  void* rec;
  size_t tree_elems = 0;
  double* G;
  double* Ginv;
  float* Ginvf;                   // float copy of Ginv (float compute types)
  double* P;
  double* R;
  double* Rinv;
  double* Gpart;
  int gsplit = 1;
  double* rowpart;
  double* rowred;                 // grid-wide sums of the row partials of modes over 1024 points
  unsigned* bar;                  // grid-barrier words of the fused update
  unsigned* redcnt;               // last-CTA reduction counters (zero between launches)
  void* w1T;                      // w_1 in the compute type
  void* wcolT;                    // mode-1 column weights prod_{m>1} w_m in the compute type
  unsigned long long* stamps;     // phase timer stamps of the fused update (profiling)
  unsigned long long* span_dev;   // the projection kernel's span words (profiling, TcPlan::span)
  int ntile = 1;
  double* sig2;
  double* sig2_lag;               // sigma^2 of the state a step starts from (estimator features)
  int* need_scratch;              // the estimator's gate word when it does not gate
  float* Vprev;
  float* Vprev_bak;
  double* npart;
  int nblk = 256;
  Readback* rb_dev;
  unsigned* flags;
  // HOSVD scratch
  double* C64;
  void* Cc;
  void* jA;
  void* jV;
  void* siQ;
  void* siZ;
  void* siX;
  double* siG;
  double* siR;
  void* siH;
  void* siJA;
  void* siJV;
  double* wpart;
  float* eigf;                    // float eigensolver scratch (float compute types)
  float* wsf[kMaxModes];          // sqrt of the weights in float
  size_t wpart_cap = 0;
  double* ev[kMaxModes];
  double* Qeig[kMaxModes];
  double* trace;
  double* eigscratch;
  double* Zs;                     // eigenvectors of the short-side Gram of a long mode (M x kcap)
  double* wq;                     // merged weights of the other modes and their square roots (2 M)
  // BF16 tensor-core projection
  TcPlan tc;
  bool use_tc = false;
  // learned error estimator
  EstState est;
  float* mlpP = nullptr;
  float* mlpNorm = nullptr;
  float* mlpM = nullptr;
  float* mlpV = nullptr;
  float* mlpG = nullptr;
  float* mlpGpart = nullptr;
  float* mlpLpart = nullptr;
  float* mlpLoss = nullptr;
  float* trX = nullptr;
  float* trT = nullptr;
  int mlp_parts = 128;
  int tr_cap = 8192;
  // recorded (features, target) rows: the last tr_cap rows from tr_off on (the rows before
  // tr_off are dropped in one move once they number tr_cap, so each row costs O(1))
  std::vector<float> hX, hT;
  size_t tr_off = 0;
  // profiling (CUDA events on the stream)
  bool prof = false;
  cudaEvent_t pev[6] = {nullptr};
  tdb_profile pacc;

  // pinned host staging: the step record read back each step and the estimator state /
  // error gate sent down each step (copies that stream capture can record)
  Readback* rb_pin = nullptr;
  EstState* est_pin = nullptr;
  int* need_pin = nullptr;
  const EstState* est_pin_d = nullptr;   // device views of the pinned words (null: copies instead)
  const int* need_pin_d = nullptr;
  EstState* est_dev = nullptr;
  bool need_host = false;          // this step's host gate (evaluate the exact error)
  bool gated_step = false;         // the estimator decides on the device this step
  // input slots and the captured step graphs (one per slot parity)
  const void* slot[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  uint64_t gkey[2] = {0, 0};
  long long gcount[2] = {0, 0};     // library kernels recorded in each graph (launch counter)
  cudaStream_t cap_stream = nullptr; // steps are recorded here (any stream can replay them)
  cudaStream_t aux = nullptr;        // second branch of a step (G_n refresh beside the exact error)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool graph_broken = false;
  bool prof_graph_ok = true;      // profiled steps may be recorded (their events time in a graph)
  bool last_graphed = false;      // the step being finished ran as a graph replay
  bool main_from_start = false;   // its projection kernel is timed from the step's first event
  int64_t graph_replays = 0, graph_records = 0;
  // steps of tdb_push_snapshot, recorded per (V_{k+1}, V_k, V_{k-1}) pointer tuple once
  // the tuple recurs (a ring of input buffers); tuples seen once run eagerly
  struct PtrGraph {
    const void* v[3];
    uint64_t key;
    cudaGraphExec_t exec;
    long long count;
    uint64_t used;
  };
  static constexpr int kPtrGraphs = 6, kPtrSeen = 8;
  PtrGraph pgraph[kPtrGraphs] = {};
  const void* pseen[kPtrSeen][3] = {};
  int pseen_next = 0;
  uint64_t ptick = 0;

  // host state
  const void* V_prev = nullptr;
  const void* V_prev2 = nullptr;   // the snapshot before V_prev (central differences), or null
  bool ready = false;
  bool warm = false;
  int64_t step = 0, reinits = 0, exact_evals = 0;
  std::vector<double> history;
  Readback rb;
  std::vector<double> h_ev[kMaxModes];
  double h_trace[kMaxModes];

  ~tdb_ctx() {
    for (int i = 0; i < 2; ++i)
      if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
    for (auto& g : pgraph)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (aux) cudaStreamDestroy(aux);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (rb_pin) cudaFreeHost(rb_pin);
  }
};

struct tdb_batch {
  std::vector<tdb_ctx*> m;
  cudaStream_t main = nullptr;       // the caller's stream: graphs are launched here
  cudaStream_t cap = nullptr;        // private origin stream of the recording
  std::vector<cudaStream_t> st;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<uint64_t> keys[2];
  long long gcount[2] = {0, 0};
  bool broken = false;
  int64_t replays = 0, records = 0;
  std::string err;

  ~tdb_batch() {
    for (int i = 0; i < 2; ++i)
      if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
    for (auto e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (auto q : st) cudaStreamDestroy(q);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
      return TDB_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define CHECK_LAUNCH()                                                                  \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) {                                                            \
      ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e_);              \
      return TDB_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define TRY(x)                            \
  do {                                    \
    tdb_status s_ = (x);                  \
    if (s_ != TDB_OK) return s_;          \
  } while (0)

// A mode of more points than this (the first or the last, the others' product at most this)
// takes its HOSVD from the short side: the Gram of the other modes' merged index.
constexpr int64_t kDirectGramMax = 1024;
bool short_side(const tdb_ctx* c, int n) { return c->N[n] > kDirectGramMax; }
int64_t gram_dim(const tdb_ctx* c, int n) { return short_side(c, n) ? c->S / c->N[n] : c->N[n]; }

int64_t prod_except(const int64_t* a, int p, int n) {
  int64_t v = 1;
  for (int m = 0; m < p; ++m)
    if (m != n) v *= a[m];
  return v;
}

std::vector<int> clamp_product_bound(std::vector<int> r) {
  bool changed = true;
  int p = (int)r.size();
  while (changed) {
    changed = false;
    for (int n = 0; n < p; ++n) {
      int64_t other = 1;
      for (int m = 0; m < p; ++m)
        if (m != n) other *= r[m];
      if (r[n] > other) {
        r[n] = (int)other;
        changed = true;
      }
    }
  }
  return r;
}

// Smallest r with sum_{i<=r} max(lambda_i, 0) >= gamma/100 * total (Eq. 2.21, first form).
int rank_from_spectrum(const std::vector<double>& lam, double total, double gamma_th) {
  if (!(total > 0.0)) return 1;
  double target = gamma_th / 100.0 * total, acc = 0.0;
  for (size_t i = 0; i < lam.size(); ++i) {
    acc += std::max(lam[i], 0.0);
    if (acc >= target) return (int)i + 1;
  }
  return (int)lam.size() + 1;
}

// Smallest r with sum_{i<=r} sigma_i^2 >= gamma/100 (sum sigma^2 + eps^2) (Eq. 2.21, second form).
int rank_from_core(const double* s2, int r, double eps, double gamma_th) {
  double denom = eps * eps;
  for (int i = 0; i < r; ++i) denom += std::max(s2[i], 0.0);
  double target = gamma_th / 100.0 * denom, acc = 0.0;
  for (int i = 0; i < r; ++i) {
    acc += std::max(s2[i], 0.0);
    if (acc >= target) return i + 1;
  }
  return r;
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
void carve(tdb_ctx* c, Carver& cv) {
  const int p = c->p;
  const size_t tsz = c->f64 ? 8 : 4;
  int64_t Rprod = 1;
  for (int n = 0; n < p; ++n) Rprod *= c->cap[n];
  int64_t Nmax = 0, Ng = 0;   // longest mode; largest Gram the HOSVD forms
  for (int n = 0; n < p; ++n) Nmax = std::max<int64_t>(Nmax, c->N[n]);
  for (int n = 0; n < p; ++n) Ng = std::max<int64_t>(Ng, gram_dim(c, n));
  for (int n = 0; n < p; ++n) {
    int64_t nr = c->N[n] * c->cap[n];
    c->w[n] = cv.take<double>(c->N[n]);
    c->U[n] = cv.take<double>(nr);
    c->Up[n] = cv.take<double>(nr);
    c->X[n] = cv.take<double>(nr);
    c->Ubak[n] = cv.take<double>(nr);
    c->A[n] = cv.take<char>(nr * tsz);
    c->Uc[n] = cv.take<char>(nr * tsz);
    int64_t ysz = c->N[n] * (Rprod / c->cap[n]);
    c->Y[n] = cv.take<char>(ysz * tsz);
  }
  c->T = cv.take<double>(Rprod);
  c->T2 = cv.take<double>(Rprod);
  c->Tbak = cv.take<double>(Rprod);
  c->Tcore = c->f64 ? (void*)c->T : (void*)cv.take<char>(Rprod * tsz);
  c->dS = cv.take<char>(Rprod * tsz);
  // tree scratch: the largest intermediate of the projection or reconstruction chains
  int64_t tree = 0;
  for (int n = 0; n < p; ++n) tree = std::max<int64_t>(tree, c->S / c->N[n] * c->cap[n]);
  tree = std::max<int64_t>(tree, Rprod);
  c->tree_elems = tree;
  c->ping = cv.take<char>(tree * tsz);
  c->pong = cv.take<char>(tree * tsz);
  c->dV = cv.take<char>(c->S * tsz);
  c->rec = cv.take<char>(c->S * tsz);
  c->G = cv.take<double>(p * kMaxRank * kMaxRank);
  c->Ginv = cv.take<double>(p * kMaxRank * kMaxRank);
  c->Ginvf = c->f64 ? nullptr : cv.take<float>(p * kMaxRank * kMaxRank);
  c->P = cv.take<double>(p * kMaxRank * kMaxRank);
  c->R = cv.take<double>(p * kMaxRank * kMaxRank);
  c->Rinv = cv.take<double>(p * kMaxRank * kMaxRank);
  c->gsplit = 64;
  c->Gpart = cv.take<double>((size_t)p * c->gsplit * kMaxRank * kMaxRank);
  c->ntile = (int)((Nmax + 31) / 32);
  c->rowpart = cv.take<double>((size_t)2 * p * c->ntile * kMaxRank * kMaxRank);
  c->rowred = cv.take<double>((size_t)2 * kMaxModes * kMaxRank * kMaxRank);
  c->bar = cv.take<unsigned>(2);
  c->redcnt = cv.take<unsigned>(8);
  c->w1T = cv.take<char>((size_t)c->N[0] * tsz);
  c->wcolT = cv.take<char>((size_t)(c->S / c->N[0]) * tsz);
  c->stamps = cv.take<unsigned long long>(32);
  c->span_dev = cv.take<unsigned long long>(4);
  c->sig2 = cv.take<double>(p * kMaxRank);
  c->sig2_lag = cv.take<double>(p * kMaxRank);
  c->need_scratch = cv.take<int>(1);
  c->Vprev = cv.take<float>(p * kMaxRank * kMaxRank);
  c->Vprev_bak = cv.take<float>(p * kMaxRank * kMaxRank);
  c->nblk = 608;
  c->npart = cv.take<double>(c->nblk);
  c->rb_dev = cv.take<Readback>(1);
  c->est_dev = cv.take<EstState>(1);
  c->flags = &c->rb_dev->flags;
  // HOSVD scratch (sized by the Gram dimension: N_n, or the short side of a long mode)
  int64_t nn = (Ng + 1) & ~1;
  c->C64 = cv.take<double>(Ng * Ng);
  c->Cc = cv.take<char>(Ng * Ng * tsz);
  // eigensolver blocks: double in every compute type (float contexts refine in double)
  int64_t nsmall = std::min<int64_t>(nn, 96);
  c->jA = cv.take<double>(nsmall * nsmall);
  c->jV = cv.take<double>(nsmall * nsmall);
  c->siQ = cv.take<double>(Ng * 64);
  c->siZ = cv.take<double>(Ng * 64);
  c->siX = cv.take<double>(Ng * 64);
  c->siG = cv.take<double>(64 * 64);
  c->siR = cv.take<double>(64 * 64);
  c->siH = cv.take<double>(64 * 64);
  c->siJA = cv.take<double>(64 * 64);
  c->siJV = cv.take<double>(64 * 64);
  int ntile = (int)((Ng + 31) / 32);
  c->wpart_cap = std::max<size_t>((size_t)(ntile * (ntile + 1) / 2) * 8 * 1024, (size_t)152 * 64 * 64);
  c->wpart = cv.take<double>(c->wpart_cap);
  c->eigf = c->f64 ? nullptr : cv.take<float>(eig_si_scratch_floats((int)Ng));
  for (int n = 0; n < p; ++n) c->wsf[n] = c->f64 ? nullptr : cv.take<float>(c->N[n]);
  for (int n = 0; n < p; ++n) {
    c->kcap[n] = (int)std::min<int64_t>(gram_dim(c, n), c->cap[n] + 2);
    c->ev[n] = cv.take<double>(c->kcap[n]);
    c->Qeig[n] = cv.take<double>(c->N[n] * c->kcap[n]);
  }
  c->trace = cv.take<double>(p);
  int kmax = 0;
  for (int n = 0; n < p; ++n) kmax = std::max(kmax, c->kcap[n]);
  c->eigscratch = cv.take<double>(64 + Ng * (kmax + 2));
  c->Zs = cv.take<double>(Ng * kmax);
  c->wq = cv.take<double>(2 * Ng);
  c->mlpP = cv.take<float>(MLP_NPARAM);
  c->mlpNorm = cv.take<float>(2 * MLP_F + 2);
  c->mlpM = cv.take<float>(MLP_NPARAM);
  c->mlpV = cv.take<float>(MLP_NPARAM);
  c->mlpG = cv.take<float>(MLP_NPARAM);
  c->mlpGpart = cv.take<float>((size_t)c->mlp_parts * MLP_NPARAM);
  c->mlpLpart = cv.take<float>(c->mlp_parts);
  c->mlpLoss = cv.take<float>(1);
  c->trX = cv.take<float>((size_t)c->tr_cap * MLP_F);
  c->trT = cv.take<float>(c->tr_cap);
  if (c->prec == TDB_BF16_TTM) tc_carve(c->tc, cv, c->p, c->N, c->cap);
}

tdb_status validate(const tdb_config* cfg, std::string& err) {
  if (!cfg) { err = "null config"; return TDB_ERR_INVALID_ARG; }
  if (cfg->ndim < 2 || cfg->ndim > kMaxModes) { err = "ndim must be 2..4"; return TDB_ERR_SHAPE; }
  {
    int64_t S = 1;
    for (int n = 0; n < cfg->ndim; ++n) {
      if (cfg->dims[n] < 1 || cfg->dims[n] >= ((int64_t)1 << 31)) { err = "mode sizes must be positive"; return TDB_ERR_SHAPE; }
      S *= cfg->dims[n];
      if (S >= ((int64_t)1 << 31)) { err = "a snapshot must have fewer than 2^31 elements"; return TDB_ERR_SHAPE; }
    }
    for (int n = 0; n < cfg->ndim; ++n)
      if (cfg->dims[n] > kDirectGramMax && ((n != 0 && n != cfg->ndim - 1) || S / cfg->dims[n] > kDirectGramMax)) {
        err = "a mode of more than 1024 points must be the first or the last, and the other modes at most 1024 "
              "points together";
        return TDB_ERR_SHAPE;
      }
  }
  if (cfg->precision < TDB_FP64 || cfg->precision > TDB_BF16_TTM) { err = "bad precision"; return TDB_ERR_INVALID_ARG; }
  if (cfg->error_mode < TDB_ERRMODE_EXACT || cfg->error_mode > TDB_ERRMODE_NONE) {
    err = "bad error_mode";
    return TDB_ERR_INVALID_ARG;
  }
  if (cfg->integrator < TDB_EULER || cfg->integrator > TDB_RK2_CENTRAL) { err = "bad integrator"; return TDB_ERR_INVALID_ARG; }
  if (cfg->eps_th > 0 && !(cfg->gamma_th > 0 && cfg->gamma_th <= 100)) { err = "gamma_th must be in (0, 100]"; return TDB_ERR_INVALID_ARG; }
  for (int n = 0; n < cfg->ndim; ++n) {
    if (cfg->rank[n] < 0 || cfg->rank[n] > kMaxRank) { err = "rank outside 0..32"; return TDB_ERR_RANK; }
    if (cfg->rank_max[n] < 0 || cfg->rank_max[n] > kMaxRank) { err = "rank_max outside 0..32"; return TDB_ERR_RANK; }
  }
  return TDB_OK;
}

void setup_dims(tdb_ctx* c, const tdb_config* cfg) {
  c->cfg = *cfg;
  c->p = cfg->ndim;
  c->S = 1;
  for (int n = 0; n < c->p; ++n) {
    c->N[n] = cfg->dims[n];
    c->S *= c->N[n];
  }
  if (c->cfg.slope_window <= 0) c->cfg.slope_window = 10;
  if (c->cfg.error_every <= 0) c->cfg.error_every = 1;
  c->prec = cfg->precision;
  c->f64 = (cfg->precision == TDB_FP64);
  c->esz = c->f64 ? 8 : 4;
  for (int n = 0; n < c->p; ++n) {
    int64_t rm = cfg->rank_max[n] > 0 ? cfg->rank_max[n] : kMaxRank;
    int64_t cp = std::min<int64_t>(std::min<int64_t>(rm, c->N[n]), prod_except(c->N, c->p, n));
    if (cfg->rank[n] > cp) cp = std::min<int64_t>(cfg->rank[n], std::min<int64_t>(c->N[n], kMaxRank));
    c->cap[n] = (int)std::min<int64_t>(cp, kMaxRank);
  }
}

ModeDesc mode_desc(const tdb_ctx* c) {
  ModeDesc d;
  d.p = c->p;
  for (int n = 0; n < kMaxModes; ++n) {
    d.N[n] = n < c->p ? c->N[n] : 1;
    d.r[n] = n < c->p ? c->r[n] : 1;
  }
  return d;
}

WeightView weight_view(const tdb_ctx* c) {
  WeightView wv;
  wv.p = c->p;
  for (int n = 0; n < kMaxModes; ++n) {
    wv.N[n] = n < c->p ? c->N[n] : 1;
    wv.w[n] = n < c->p ? c->w[n] : nullptr;
  }
  return wv;
}

// ---------------------------------------------------------------------------
// Projection (Eqs. 2.15, 2.16) by mode products on the unfused path
// ---------------------------------------------------------------------------
template <typename Tc>
tdb_status project_tree(tdb_ctx* ctx, const Tc* dV, cudaEvent_t* evm) {
  const int p = ctx->p;
  cudaStream_t s = ctx->stream;
  int64_t dims[kMaxModes];
  auto mp = [&](const Tc* in, Tc* out, int n, int64_t* cur) {
    int64_t L = 1, Q = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < p; ++m) Q *= cur[m];
    launch_modeprod<Tc, Tc, Tc>(in, out, (const Tc*)ctx->A[n], L, (int)cur[n], ctx->r[n], Q, ctx->N[n], 1, s);
    cur[n] = ctx->r[n];
  };
  Tc* ping = (Tc*)ctx->ping;
  Tc* pong = (Tc*)ctx->pong;
  // Z1 = dV x_1 A_1^T, then each Y_n (n >= 2) contracts the remaining modes but n
  for (int m = 0; m < p; ++m) dims[m] = ctx->N[m];
  if (evm) record_timing_event(evm[0], s);
  mp(dV, ping, 0, dims);
  if (evm) record_timing_event(evm[1], s);
  int64_t z1dims[kMaxModes];
  for (int m = 0; m < p; ++m) z1dims[m] = dims[m];
  for (int n = 1; n < p; ++n) {
    int64_t cur[kMaxModes];
    for (int m = 0; m < p; ++m) cur[m] = z1dims[m];
    std::vector<int> todo;
    for (int m = 1; m < p; ++m)
      if (m != n) todo.push_back(m);
    const Tc* src = ping;
    for (size_t t = 0; t < todo.size(); ++t) {
      Tc* dst = (t + 1 == todo.size()) ? (Tc*)ctx->Y[n] : ((t & 1) ? ping : pong);
      if (t > 0 && dst == src) dst = (dst == ping) ? pong : ping;
      if (t == 0 && todo.size() > 1) dst = pong;
      mp(src, dst, todo[t], cur);
      src = dst;
    }
    if (todo.empty()) cudaMemcpyAsync(ctx->Y[n], ping, sizeof(Tc) * ctx->S / ctx->N[0] * ctx->r[0], cudaMemcpyDeviceToDevice, s);
  }
  // Y_1 = dV x_2 A_2^T ... x_p A_p^T (ping is free again)
  {
    int64_t cur[kMaxModes];
    for (int m = 0; m < p; ++m) cur[m] = ctx->N[m];
    const Tc* src = dV;
    for (int m = 1; m < p; ++m) {
      Tc* dst = (m == p - 1) ? (Tc*)ctx->Y[0] : ((m & 1) ? ping : pong);
      mp(src, dst, m, cur);
      src = dst;
    }
  }
  // dS = Y_p x_p A_p^T
  {
    int64_t cur[kMaxModes];
    for (int m = 0; m < p; ++m) cur[m] = ctx->r[m];
    cur[p - 1] = ctx->N[p - 1];
    mp((const Tc*)ctx->Y[p - 1], (Tc*)ctx->dS, p - 1, cur);
  }
  CHECK_LAUNCH();
  return TDB_OK;
}

// V^TDB = T x_1 U_1 ... x_p U_p into out (compute type)
template <typename Tc>
tdb_status reconstruct_into(tdb_ctx* ctx, Tc* out) {
  const int p = ctx->p;
  cudaStream_t s = ctx->stream;
  int64_t cur[kMaxModes];
  for (int m = 0; m < p; ++m) cur[m] = ctx->r[m];
  const Tc* src = (const Tc*)ctx->Tcore;
  Tc* bufs[2] = {(Tc*)ctx->ping, (Tc*)ctx->pong};
  for (int n = 0; n < p; ++n) {
    Tc* dst = (n == p - 1) ? out : bufs[n & 1];
    int64_t L = 1, Q = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < p; ++m) Q *= cur[m];
    launch_modeprod<Tc, Tc, Tc>(src, dst, (const Tc*)ctx->Uc[n], L, ctx->r[n], (int)ctx->N[n], Q, 1, ctx->N[n], s);
    cur[n] = ctx->N[n];
    src = dst;
  }
  CHECK_LAUNCH();
  return TDB_OK;
}

// err2 = ||V - T x U||_W^2 (Eq. 2.20): H = T x_2 U_2 ... x_p U_p, then the fused pass
// over V that forms each mode-1 column U_1 H[:, c] on the fly.
template <typename Tc>
tdb_status exact_error2(tdb_ctx* ctx, const Tc* V, const int* gate = nullptr) {
  const int p = ctx->p;
  cudaStream_t s = ctx->stream;
  int64_t cur[kMaxModes];
  for (int m = 0; m < p; ++m) cur[m] = ctx->r[m];
  const Tc* src = (const Tc*)ctx->Tcore;
  Tc* bufs[2] = {(Tc*)ctx->ping, (Tc*)ctx->pong};
  for (int n = 1; n < p; ++n) {
    Tc* dst = bufs[n & 1];
    int64_t L = 1, Q = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < p; ++m) Q *= cur[m];
    launch_modeprod<Tc, Tc, Tc>(src, dst, (const Tc*)ctx->Uc[n], L, ctx->r[n], (int)ctx->N[n], Q, 1, ctx->N[n], s,
                                gate);
    cur[n] = ctx->N[n];
    src = dst;
  }
  launch_recon_err<Tc>(V, (const Tc*)ctx->Uc[0], src, ctx->r[0], (int)ctx->N[0], ctx->S / ctx->N[0],
                       (const Tc*)ctx->w1T, (const Tc*)ctx->wcolT, ctx->npart, ctx->redcnt, ctx->nblk,
                       &ctx->rb_dev->err2, ctx->flags, s, gate);
  CHECK_LAUNCH();
  return TDB_OK;
}

// Refresh everything derived from (T, U): compute-type copies, weighted bases,
// G_n, its inverse and sigma^(n) (Eq. 2.18).
template <typename Tc>
tdb_status refresh_derived(tdb_ctx* ctx, bool bases_too) {
  cudaStream_t s = ctx->stream;
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) Rprod *= ctx->r[n];
  if (!ctx->f64) launch_cast<double, float>(ctx->T, (float*)ctx->Tcore, Rprod, s);
  for (int n = 0; n < ctx->p; ++n) {
    if (bases_too) launch_weighted_bases<Tc>(ctx->U[n], ctx->w[n], (Tc*)ctx->A[n], ctx->N[n], ctx->r[n], s);
    if (ctx->f64)
      cudaMemcpyAsync(ctx->Uc[n], ctx->U[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToDevice, s);
    else
      launch_cast<double, float>(ctx->U[n], (float*)ctx->Uc[n], ctx->N[n] * ctx->r[n], s);
  }
  ModeDesc d = mode_desc(ctx);
  const int nsplit = gram_split(ctx->r, ctx->p, ctx->gsplit);
  launch_gram(d, ctx->T, ctx->Gpart, nsplit, ctx->G, ctx->Ginv, ctx->Ginvf, ctx->sig2, ctx->Vprev, ctx->warm ? 1 : 0, ctx->flags, s);
  ctx->warm = true;
  CHECK_LAUNCH();
  return TDB_OK;
}

// The step record: sigma^2 into the record, then the record to pinned host memory.
tdb_status readback_enqueue(tdb_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(ctx->rb_dev->sig2, ctx->sig2, sizeof(double) * ctx->p * kMaxRank, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ctx->rb_pin, ctx->rb_dev, sizeof(Readback), cudaMemcpyDeviceToHost, s));
  return TDB_OK;
}

// After the stream (or a graph holding readback_enqueue) has completed.
tdb_status readback_done(tdb_ctx* ctx) {
  ctx->rb = *ctx->rb_pin;
  if (ctx->rb.flags & kFlagTimeout) { ctx->err = "device wait timed out"; return TDB_ERR_TIMEOUT; }
  return TDB_OK;
}

tdb_status readback(tdb_ctx* ctx) {
  TRY(readback_enqueue(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  return readback_done(ctx);
}

// ---------------------------------------------------------------------------
// HOSVD: per-mode spectrum (leading eigenpairs and trace), then the truncated state
// ---------------------------------------------------------------------------
// Spectrum and leading eigenvectors of C_n for a long first or last mode n from the short
// side: K, the weighted Gram of the other modes' merged index (M x M, M = S / N_n), has the
// nonzero eigenvalues of C_n, and its unit eigenvector z maps to C_n's as B z / sqrt(lambda)
// (B the weighted unfolding; the thin SVD of B).  Float compute types read the weighted
// data in ctx->rec and solve in double as for the direct route.
template <typename Tc>
tdb_status hosvd_short(tdb_ctx* ctx, const Tc* V, int n) {
  cudaStream_t s = ctx->stream;
  const int64_t Nn = ctx->N[n], M = ctx->S / Nn;
  const int first = (n == 0) ? 1 : 0;
  const int k = ctx->kcap[n], Mi = (int)M;
  tdb_status st;
  if (!ctx->f64) {
    launch_gram_weighted((const float*)ctx->rec, first ? Nn : 1, M, first ? 1 : Nn, ctx->wpart, ctx->wpart_cap,
                         ctx->C64, (float*)ctx->Cc, s);
    CHECK_LAUNCH();
    if (Mi <= 48) {
      st = eig_leading_small<double>(ctx->C64, ctx->C64, Mi, k, (double*)ctx->jA, (double*)ctx->jV, ctx->flags,
                                     ctx->ev[n], ctx->Zs, ctx->trace + n, ctx->eigscratch, s);
    } else {
      st = eig_si_float((const float*)ctx->Cc, ctx->C64, Mi, k, 24, ctx->eigf, ctx->bar, ctx->flags, ctx->ev[n],
                        ctx->Zs, ctx->trace + n, s);
      if (st == TDB_OK) {
        SubspaceWs<double> ws{(double*)ctx->siQ, (double*)ctx->siZ, (double*)ctx->siX, ctx->siG, ctx->siR,
                              (double*)ctx->siH, (double*)ctx->siJA, (double*)ctx->siJV};
        st = eig_subspace<double>(ctx->C64, ctx->C64, Mi, k, 3, ws, ctx->flags, ctx->ev[n], ctx->Zs, ctx->trace + n,
                                  ctx->eigscratch, s, ctx->Zs);
      }
    }
    if (st != TDB_OK) { ctx->err = "eigensolver launch failed"; return st; }
    launch_short_map<float>((const float*)ctx->rec, first, Nn, M, nullptr, nullptr, ctx->Zs, ctx->ev[n], k,
                            ctx->Qeig[n], s);
  } else {
    launch_merge_weights(weight_view(ctx), n, M, ctx->wq, s);
    // K as the mode Gram of a two-mode view: (N_n, M) for the first mode, (M, N_n) for the last
    GramView g;
    g.p = 2;
    g.n = first;
    for (int m = 0; m < kMaxModes; ++m) { g.N[m] = 1; g.w[m] = nullptr; }
    g.N[first ? 0 : 1] = Nn;
    g.w[first ? 0 : 1] = ctx->w[n];
    g.N[first ? 1 : 0] = M;
    g.w[first ? 1 : 0] = ctx->wq;
    g.Nn = M;
    g.L = first ? Nn : 1;
    g.Q = first ? 1 : Nn;
    launch_wgram<Tc>(V, g, ctx->wpart, ctx->wpart_cap, ctx->C64, ctx->Cc, 0, s);
    CHECK_LAUNCH();
    if (Mi <= 96) {
      st = eig_leading_small<Tc>((const Tc*)ctx->Cc, ctx->C64, Mi, k, (Tc*)ctx->jA, (Tc*)ctx->jV, ctx->flags,
                                 ctx->ev[n], ctx->Zs, ctx->trace + n, ctx->eigscratch, s);
    } else {
      SubspaceWs<Tc> ws{(Tc*)ctx->siQ, (Tc*)ctx->siZ, (Tc*)ctx->siX, ctx->siG, ctx->siR,
                        (Tc*)ctx->siH, (Tc*)ctx->siJA, (Tc*)ctx->siJV};
      st = eig_subspace<Tc>((const Tc*)ctx->Cc, ctx->C64, Mi, k, 24, ws, ctx->flags, ctx->ev[n], ctx->Zs,
                            ctx->trace + n, ctx->eigscratch, s);
    }
    if (st != TDB_OK) { ctx->err = "eigensolver launch failed"; return st; }
    launch_short_map<Tc>(V, first, Nn, M, ctx->w[n], ctx->wq + M, ctx->Zs, ctx->ev[n], k, ctx->Qeig[n], s);
  }
  CHECK_LAUNCH();
  return TDB_OK;
}

template <typename Tc>
tdb_status hosvd_spectrum(tdb_ctx* ctx, const Tc* V) {
  cudaStream_t s = ctx->stream;
  if (!ctx->f64) {
    // float compute types: weight the data once, 64 x 64 Gram tiles, cooperative eigensolver
    for (int n = 0; n < ctx->p; ++n) launch_sqrt_weights(ctx->w[n], (int)ctx->N[n], ctx->wsf[n], s);
    launch_weight_data((const float*)V, ctx->p, ctx->N, ctx->wsf, ctx->S, (float*)ctx->rec, s);
    CHECK_LAUNCH();
    for (int n = 0; n < ctx->p; ++n) {
      if (short_side(ctx, n)) {
        TRY(hosvd_short<Tc>(ctx, V, n));
        continue;
      }
      int64_t L = 1, Q = 1;
      for (int m = 0; m < n; ++m) L *= ctx->N[m];
      for (int m = n + 1; m < ctx->p; ++m) Q *= ctx->N[m];
      launch_gram_weighted((const float*)ctx->rec, L, ctx->N[n], Q, ctx->wpart, ctx->wpart_cap, ctx->C64,
                           (float*)ctx->Cc, s);
      CHECK_LAUNCH();
      const int Nn = (int)ctx->N[n];
      tdb_status st;
      // The Gram is accurate to about 1e-9 of its largest entries (float products,
      // float-float sums), but a float eigensolver resolves eigenvectors only where the
      // eigenvalue gaps exceed about 1e-6 of the largest eigenvalue; the eigenvectors the
      // rank rule keeps at gamma_th = 99.999 % sit below that.  So the solve is double: the
      // single-CTA Jacobi on the double Gram for short modes, and for long ones the float
      // subspace iteration as a warm start refined by three double iterations with
      // Rayleigh-Ritz.
      if (Nn <= 48) {
        st = eig_leading_small<double>(ctx->C64, ctx->C64, Nn, ctx->kcap[n], (double*)ctx->jA, (double*)ctx->jV,
                                       ctx->flags, ctx->ev[n], ctx->Qeig[n], ctx->trace + n, ctx->eigscratch, s);
      } else {
        st = eig_si_float((const float*)ctx->Cc, ctx->C64, Nn, ctx->kcap[n], 24, ctx->eigf, ctx->bar, ctx->flags,
                          ctx->ev[n], ctx->Qeig[n], ctx->trace + n, s);
        if (st == TDB_OK) {
          SubspaceWs<double> ws{(double*)ctx->siQ, (double*)ctx->siZ, (double*)ctx->siX, ctx->siG, ctx->siR,
                                (double*)ctx->siH, (double*)ctx->siJA, (double*)ctx->siJV};
          st = eig_subspace<double>(ctx->C64, ctx->C64, Nn, ctx->kcap[n], 3, ws, ctx->flags, ctx->ev[n],
                                    ctx->Qeig[n], ctx->trace + n, ctx->eigscratch, s, ctx->Qeig[n]);
        }
      }
      if (st != TDB_OK) { ctx->err = "eigensolver launch failed"; return st; }
      CHECK_LAUNCH();
    }
  } else
  for (int n = 0; n < ctx->p; ++n) {
    if (short_side(ctx, n)) {
      TRY(hosvd_short<Tc>(ctx, V, n));
      continue;
    }
    GramView g;
    g.p = ctx->p;
    g.n = n;
    for (int m = 0; m < kMaxModes; ++m) {
      g.N[m] = m < ctx->p ? ctx->N[m] : 1;
      g.w[m] = m < ctx->p ? ctx->w[m] : nullptr;
    }
    g.Nn = ctx->N[n];
    g.L = 1;
    for (int m = 0; m < n; ++m) g.L *= ctx->N[m];
    g.Q = 1;
    for (int m = n + 1; m < ctx->p; ++m) g.Q *= ctx->N[m];
    launch_wgram<Tc>(V, g, ctx->wpart, ctx->wpart_cap, ctx->C64, ctx->Cc, ctx->f64 ? 0 : 1, s);
    CHECK_LAUNCH();
    int Nn = (int)ctx->N[n];
    tdb_status st;
    if (Nn <= 96)
      st = eig_leading_small<Tc>((const Tc*)ctx->Cc, ctx->C64, Nn, ctx->kcap[n], (Tc*)ctx->jA, (Tc*)ctx->jV,
                                 ctx->flags, ctx->ev[n], ctx->Qeig[n], ctx->trace + n, ctx->eigscratch, s);
    else {
      SubspaceWs<Tc> ws{(Tc*)ctx->siQ, (Tc*)ctx->siZ, (Tc*)ctx->siX, ctx->siG, ctx->siR,
                        (Tc*)ctx->siH, (Tc*)ctx->siJA, (Tc*)ctx->siJV};
      st = eig_subspace<Tc>((const Tc*)ctx->Cc, ctx->C64, Nn, ctx->kcap[n], 24, ws, ctx->flags, ctx->ev[n],
                            ctx->Qeig[n], ctx->trace + n, ctx->eigscratch, s);
    }
    if (st != TDB_OK) { ctx->err = "eigensolver launch failed"; return st; }
    CHECK_LAUNCH();
  }
  // spectrum to host (needed by the rank rule)
  for (int n = 0; n < ctx->p; ++n) {
    ctx->h_ev[n].resize(ctx->kcap[n]);
    CK(cudaMemcpyAsync(ctx->h_ev[n].data(), ctx->ev[n], sizeof(double) * ctx->kcap[n], cudaMemcpyDeviceToHost, s));
  }
  CK(cudaMemcpyAsync(ctx->h_trace, ctx->trace, sizeof(double) * ctx->p, cudaMemcpyDeviceToHost, s));
  unsigned fl = 0;
  CK(cudaMemcpyAsync(&fl, ctx->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (fl & kFlagTimeout) { ctx->err = "eigensolver wait timed out"; return TDB_ERR_TIMEOUT; }
  return TDB_OK;
}

template <typename Tc>
tdb_status hosvd_state(tdb_ctx* ctx, const Tc* V, const int* ranks) {
  cudaStream_t s = ctx->stream;
  for (int n = 0; n < ctx->p; ++n) ctx->r[n] = ranks[n];
  // U_n = W^{-1/2} Q_n[:, :r_n], then weighted Cholesky-QR so that U^T W U = I in double
  for (int n = 0; n < ctx->p; ++n) launch_scale_basis(ctx->Qeig[n], ctx->w[n], ctx->N[n], ctx->r[n], ctx->Up[n], s);
  RowArgs a;
  memset(&a, 0, sizeof(a));
  a.d = mode_desc(ctx);
  for (int n = 0; n < ctx->p; ++n) {
    a.U[n] = ctx->U[n];
    a.w[n] = ctx->w[n];
    a.Up[n] = ctx->Up[n];
    a.Uout[n] = ctx->U[n];
    a.A[n] = ctx->A[n];
  }
  a.part = ctx->rowpart;
  a.ntile = ctx->ntile;
  launch_orthonormalize<Tc>(a, ctx->R, ctx->Rinv, ctx->flags, s);
  CHECK_LAUNCH();
  // T = V x_1 A_1^T ... x_p A_p^T  (Eq. 2.15 projection applied to V)
  int64_t cur[kMaxModes];
  for (int m = 0; m < ctx->p; ++m) cur[m] = ctx->N[m];
  const Tc* src = V;
  Tc* bufs[2] = {(Tc*)ctx->ping, (Tc*)ctx->pong};
  for (int n = 0; n < ctx->p; ++n) {
    Tc* dst = bufs[n & 1];
    int64_t L = 1, Q = 1;
    for (int m = 0; m < n; ++m) L *= cur[m];
    for (int m = n + 1; m < ctx->p; ++m) Q *= cur[m];
    launch_modeprod<Tc, Tc, Tc>(src, dst, (const Tc*)ctx->A[n], L, (int)cur[n], ctx->r[n], Q, ctx->N[n], 1, s);
    cur[n] = ctx->r[n];
    src = dst;
  }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) Rprod *= ctx->r[n];
  if (ctx->f64)
    CK(cudaMemcpyAsync(ctx->T, src, sizeof(double) * Rprod, cudaMemcpyDeviceToDevice, s));
  else
    launch_cast<float, double>((const float*)src, ctx->T, Rprod, s);
  CHECK_LAUNCH();
  ctx->warm = false;
  return refresh_derived<Tc>(ctx, false);
}

// Copy / restore the state for the revert guard of the rank-reduction rule.
tdb_status backup_state(tdb_ctx* ctx, int* rsave) {
  cudaStream_t s = ctx->stream;
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) { Rprod *= ctx->r[n]; rsave[n] = ctx->r[n]; }
  CK(cudaMemcpyAsync(ctx->Tbak, ctx->T, sizeof(double) * Rprod, cudaMemcpyDeviceToDevice, s));
  for (int n = 0; n < ctx->p; ++n)
    CK(cudaMemcpyAsync(ctx->Ubak[n], ctx->U[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ctx->Vprev_bak, ctx->Vprev, sizeof(float) * ctx->p * kMaxRank * kMaxRank, cudaMemcpyDeviceToDevice, s));
  return TDB_OK;
}

template <typename Tc>
tdb_status restore_state(tdb_ctx* ctx, const int* rsave) {
  cudaStream_t s = ctx->stream;
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) { ctx->r[n] = rsave[n]; Rprod *= ctx->r[n]; }
  CK(cudaMemcpyAsync(ctx->T, ctx->Tbak, sizeof(double) * Rprod, cudaMemcpyDeviceToDevice, s));
  for (int n = 0; n < ctx->p; ++n)
    CK(cudaMemcpyAsync(ctx->U[n], ctx->Ubak[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ctx->Vprev, ctx->Vprev_bak, sizeof(float) * ctx->p * kMaxRank * kMaxRank, cudaMemcpyDeviceToDevice, s));
  ctx->warm = true;
  return refresh_derived<Tc>(ctx, true);
}

template <typename Tc>
tdb_status error_now(tdb_ctx* ctx, const Tc* V, double* eps) {
  TRY(exact_error2<Tc>(ctx, V));
  TRY(readback(ctx));
  *eps = std::sqrt(std::max(ctx->rb.err2, 0.0));
  ctx->exact_evals++;
  return TDB_OK;
}

// Exact error of a freshly initialised state: seeds the estimator's last error.
template <typename Tc>
tdb_status seed_estimator(tdb_ctx* ctx, const Tc* V) {
  double e;
  TRY(error_now<Tc>(ctx, V, &e));
  ctx->exact_evals--;               // not a step's evaluation
  ctx->est.last_log_eps = std::log10(std::max(e, 1e-300));
  return TDB_OK;
}

// Largest discarded HOSVD energy among modes below their caps (lowest mode on ties, fractions
// within 1e-9 relative + 1e-12 counting as tied),
// then other modes follow until r_n <= prod_{m != n} r_m holds.
bool raise_one(tdb_ctx* ctx, const std::vector<int>& r, std::vector<int>& out) {
  auto disc = [&](int n, int rn) {
    double tot = ctx->h_trace[n];
    double kept = 0.0;
    for (int i = 0; i < rn && i < (int)ctx->h_ev[n].size(); ++i) kept += std::max(ctx->h_ev[n][i], 0.0);
    return tot > 0 ? 1.0 - kept / tot : 0.0;
  };
  out = r;
  auto pick = [&](int exclude) {
    int best = -1;
    double bv = -1.0;
    for (int n = 0; n < ctx->p; ++n) {
      if (n == exclude || out[n] >= ctx->cap[n]) continue;
      double d = disc(n, out[n]);
      // a later mode wins only by more than rounding: discarded fractions within 1e-9
      // relative + 1e-12 are tied (equal spectra of a symmetric field)
      if (best < 0 || d > bv * (1.0 + 1e-9) + 1e-12) { bv = d; best = n; }
    }
    return best;
  };
  int n0 = pick(-1);
  if (n0 < 0) return false;
  out[n0] += 1;
  while (clamp_product_bound(out) != out) {
    int m = pick(n0);
    if (m < 0) return false;
    out[m] += 1;
  }
  return true;
}

// The add/remove-mode rule of Sec. 2.5 (see tdb.h and the design notes for the reading).
template <typename Tc>
tdb_status control(tdb_ctx* ctx, const Tc* V, double eps, double* eps_after, int* n_re, int* action) {
  *eps_after = eps;
  *n_re = 0;
  *action = ACT_NONE;
  const tdb_config& cfg = ctx->cfg;
  if (cfg.eps_th <= 0) return TDB_OK;
  const int p = ctx->p, K = cfg.slope_window;
  std::vector<int> r(ctx->r, ctx->r + p);
  if (eps > cfg.eps_th) {
    TRY(hosvd_spectrum<Tc>(ctx, V));
    TRY(hosvd_state<Tc>(ctx, V, r.data()));
    double e1;
    TRY(error_now<Tc>(ctx, V, &e1));
    int nre = 1, act = ACT_REINIT;
    while (e1 > cfg.eps_th) {
      std::vector<int> nw(p);
      for (int n = 0; n < p; ++n)
        nw[n] = std::min(ctx->cap[n], std::max(r[n], rank_from_spectrum(ctx->h_ev[n], ctx->h_trace[n], cfg.gamma_th)));
      nw = clamp_product_bound(nw);
      if (nw == r) {
        std::vector<int> up;
        if (!raise_one(ctx, r, up)) { act = ACT_CAP; break; }
        nw = up;
      }
      r = nw;
      TRY(hosvd_state<Tc>(ctx, V, r.data()));
      TRY(error_now<Tc>(ctx, V, &e1));
      ++nre;
      act = ACT_INCREASE;
    }
    ctx->history.clear();
    ctx->reinits += nre;
    *eps_after = e1;
    *n_re = nre;
    *action = act;
    return TDB_OK;
  }
  ctx->history.push_back(eps);
  if ((int)ctx->history.size() > K + 1) ctx->history.erase(ctx->history.begin(), ctx->history.end() - (K + 1));
  bool excess = false;
  for (int n = 0; n < p; ++n)
    if (rank_from_core(ctx->rb.sig2[n], r[n], eps, cfg.gamma_th) < r[n]) excess = true;
  if ((int)ctx->history.size() == K + 1 && excess) {
    double slope = (ctx->history.back() - ctx->history.front()) / K;
    if (slope < 0) {
      ctx->history.clear();
      TRY(hosvd_spectrum<Tc>(ctx, V));
      std::vector<int> nw(p);
      for (int n = 0; n < p; ++n)
        nw[n] = std::min(r[n], rank_from_spectrum(ctx->h_ev[n], ctx->h_trace[n], cfg.gamma_th));
      nw = clamp_product_bound(nw);
      if (nw == r) return TDB_OK;
      int rsave[kMaxModes];
      TRY(backup_state(ctx, rsave));
      TRY(hosvd_state<Tc>(ctx, V, nw.data()));
      double e2;
      TRY(error_now<Tc>(ctx, V, &e2));
      ctx->reinits += 1;
      *n_re = 1;
      if (e2 <= cfg.eps_th) {
        *eps_after = e2;
        *action = ACT_DECREASE;
      } else {
        TRY(restore_state<Tc>(ctx, rsave));
        *action = ACT_REVERT;
      }
    }
  }
  return TDB_OK;
}

// ---------------------------------------------------------------------------
// One step: prepare (host), enqueue (device work, no host synchronisation, so that
// stream capture can record it), finish (host, after the step record is back).
// ---------------------------------------------------------------------------

// Host bookkeeping before the device work: counters, the error gate, and the staged
// estimator state.
void prepare_step(tdb_ctx* ctx) {
  ctx->step++;
  ctx->est.steps_since_exact += 1;
  ctx->est.steps_since_reinit += 1;
  ctx->gated_step = ctx->cfg.error_mode == TDB_ERRMODE_MLP && ctx->est.ready;
  switch (ctx->cfg.error_mode) {
    case TDB_ERRMODE_EXACT: ctx->need_host = true; break;
    case TDB_ERRMODE_EVERY_K: ctx->need_host = (ctx->step % ctx->cfg.error_every) == 0; break;
    case TDB_ERRMODE_MLP: ctx->need_host = true; break;      // the device decides when the estimator is ready
    default: ctx->need_host = false;
  }
  *ctx->est_pin = ctx->est;
  *ctx->need_pin = ctx->need_host ? 1 : 0;
}

// a1..a7 and the step record, on ctx->stream.  `all_paths` (graph capture) enqueues the
// exact-error kernels on every step, gated by the device word, so that the recorded
// work does not depend on host decisions.
// a3..a6 (and phase 7's refresh of G_n, G_n^{-1}, sigma^(n) unless skip_finish): the fused
// cooperative update on the projections in ctx->dS / ctx->Y.  combine: 0 = the increment on
// the current state; with the state of step k kept in Tbak / Ubak, 1 = Heun's second stage
// (the mean of y_k and the predicted state plus the increment), 2 = the midpoint scheme's
// second stage (y_k plus the increment taken at the midpoint state).
template <typename Tc>
tdb_status fused_update(tdb_ctx* ctx, bool reorth, bool skip_finish, int combine) {
  const int p = ctx->p;
  UpdArgs a;
  memset(&a, 0, sizeof(a));
  a.d = mode_desc(ctx);
  int64_t Rprod = 1, ntiles = 0;
  for (int n = 0; n < p; ++n) Rprod *= ctx->r[n];
  for (int n = 0; n < p; ++n) {
    a.Y[n] = ctx->Y[n];
    a.U[n] = ctx->U[n];
    a.Up[n] = ctx->Up[n];
    a.X[n] = ctx->X[n];
    a.w[n] = ctx->w[n];
    a.A[n] = ctx->A[n];
    a.Uc[n] = ctx->Uc[n];
    a.U0[n] = combine ? ctx->Ubak[n] : nullptr;
    ntiles += (ctx->N[n] + 31) / 32;
  }
  a.dS = ctx->dS;
  a.ds_y2 = ctx->use_tc ? ctx->Y[1] : nullptr;       // the projection leaves dS to phase 1
  a.dS_out = ctx->dS;
  a.T = ctx->T;
  a.T2 = ctx->T2;
  a.T0 = combine ? ctx->Tbak : nullptr;
  a.combine = combine;
  a.Tcore = ctx->Tcore;
  a.G = ctx->G;
  a.Ginv = ctx->Ginv;
  a.Ginvf = ctx->Ginvf;
  a.R = ctx->R;
  a.Rinv = ctx->Rinv;
  a.sig2 = ctx->sig2;
  a.Vprev = ctx->Vprev;
  a.part = ctx->rowpart;
  a.red = ctx->rowred;
  a.ntile = ctx->ntile;
  a.gpart = ctx->Gpart;
  a.gsplit = gram_split(ctx->r, p, ctx->gsplit);
  a.warm = ctx->warm ? 1 : 0;
  a.reorth = reorth ? 1 : 0;
  a.skip_finish = skip_finish ? 1 : 0;
  a.bar = ctx->bar;
  a.stamps = ctx->prof ? ctx->stamps : nullptr;
  a.flags = ctx->flags;
  const int64_t hint = std::max<int64_t>({ntiles, (int64_t)p * a.gsplit, Rprod / 2048});
  const tdb_status us = launch_update<Tc>(a, (int)std::min<int64_t>(hint, 1 << 20), ctx->stream);
  if (us != TDB_OK) {
    ctx->err = us == TDB_ERR_UNSUPPORTED ? "cooperative launch unsupported" : "fused update launch failed";
    return us;
  }
  CHECK_LAUNCH();
  return TDB_OK;
}

// Vpp: the snapshot before Vp (central differences of TDB_RK2_CENTRAL), or null.
template <typename Tc>
tdb_status enqueue_step(tdb_ctx* ctx, const Tc* Vn, const Tc* Vp, bool all_paths, const Tc* Vpp = nullptr) {
  cudaStream_t s = ctx->stream;
  const int p = ctx->p;
  // exact error every step, or gated by the estimator: the G_n refresh (G_n, G_n^{-1},
  // sigma^(n)) runs beside the error on the context's second stream
  const bool split = (ctx->cfg.error_mode == TDB_ERRMODE_EXACT || ctx->cfg.error_mode == TDB_ERRMODE_MLP) &&
                     ctx->aux && ctx->ev_fork && ctx->ev_join;
  cudaEvent_t* ev = ctx->prof ? ctx->pev : nullptr;
  const int scheme = ctx->cfg.integrator;
  // the step opens with one small kernel (step record cleared, host words fetched, the
  // estimator's sigma features - those of the state the step starts from - kept); an Euler
  // step's projection follows it by programmatic launch, so the projection's set-up
  // (barriers, TMEM, the first loads) overlaps it.  A profiled step launches the projection
  // plainly, so that its events bracket that kernel alone.
  const bool begin_kernel = ctx->need_pin_d && ctx->est_pin_d;
  const bool pdl = begin_kernel && ctx->use_tc && scheme == TDB_EULER && !ev;
  if (ctx->use_tc) ctx->tc.span = ev ? ctx->span_dev : nullptr;
  if (ev) CK(record_timing_event(ev[0], s));
  ctx->main_from_start = pdl;        // the projection's start event is the step's (ev[0])
  if (begin_kernel) {
    k_step_begin<<<1, 256, 0, s>>>(ctx->rb_dev, ctx->need_pin_d, ctx->est_pin_d, ctx->est_dev, ctx->sig2,
                                   ctx->sig2_lag, p * kMaxRank);
    count_launch();
  } else {
    CK(cudaMemsetAsync(ctx->rb_dev, 0, sizeof(Readback), s));
    CK(cudaMemcpyAsync(&ctx->rb_dev->need, ctx->need_pin, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->est_dev, ctx->est_pin, sizeof(EstState), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->sig2_lag, ctx->sig2, sizeof(double) * p * kMaxRank, cudaMemcpyDeviceToDevice, s));
  }
  int64_t Rprod = 1;
  for (int n = 0; n < p; ++n) Rprod *= ctx->r[n];
  // a1 + a2: difference scale (Vn - Vfrom) and its projection onto the current bases
  auto project = [&](cudaEvent_t* evm, const Tc* Vfrom, double scale, bool after_begin) -> tdb_status {
    if (ctx->use_tc) {
      TRY(tc_project(ctx->tc, (const float*)Vn, (const float*)Vfrom, ctx->p, ctx->N, ctx->r,
                     (const void* const*)ctx->A, (const double* const*)ctx->w, (float*)ctx->ping, (float*)ctx->pong,
                     (float*)ctx->dV, (float*)ctx->dS, (float* const*)ctx->Y, &ctx->rb_dev->dv2, ctx->flags, s, evm,
                     ctx->err, true, (float)scale, after_begin));
    } else {
      launch_diff<Tc>(Vn, Vfrom, (Tc*)ctx->dV, ctx->S, s, (Tc)scale);
      launch_wnorm2<Tc>((const Tc*)ctx->dV, nullptr, weight_view(ctx), ctx->npart, ctx->nblk, &ctx->rb_dev->dv2,
                        ctx->flags, s);
      CHECK_LAUNCH();
      TRY(project_tree<Tc>(ctx, (const Tc*)ctx->dV, evm));
    }
    return TDB_OK;
  };
  if (scheme == TDB_HEUN || scheme == TDB_RK2_CENTRAL) {
    // first stage: keep y_k = (T, U_n), then an Euler increment at y_k gives the
    // intermediate state in place (no re-orthonormalisation; G_n, G_n^{-1} refreshed for
    // it).  Heun: the whole step with Delta V (the predicted state).  Midpoint scheme:
    // half a step with the central difference at t_k, (V_{k+1} - V_{k-1}) / 4, or
    // (V_{k+1} - V_k) / 2 without V_{k-1}.
    CK(cudaMemcpyAsync(ctx->Tbak, ctx->T, sizeof(double) * Rprod, cudaMemcpyDeviceToDevice, s));
    for (int n = 0; n < p; ++n)
      CK(cudaMemcpyAsync(ctx->Ubak[n], ctx->U[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToDevice, s));
    if (scheme == TDB_HEUN) TRY(project(nullptr, Vp, 1.0, false));
    else if (Vpp) TRY(project(nullptr, Vpp, 0.25, false));
    else TRY(project(nullptr, Vp, 0.5, false));
    TRY(fused_update<Tc>(ctx, false, false, 0));
  }
  TRY(project(ev ? ev + 4 : nullptr, Vp, 1.0, pdl));
  if (ev) CK(record_timing_event(ev[1], s));
  // a3..a6 and the refresh of G_n, G_n^{-1}, sigma^(n): one cooperative launch (second
  // stages: the increment at the intermediate state, combined with y_k)
  TRY(fused_update<Tc>(ctx, ctx->cfg.reorth != 0, split,
                       scheme == TDB_HEUN ? 1 : (scheme == TDB_RK2_CENTRAL ? 2 : 0)));
  if (ev) CK(record_timing_event(ev[2], s));
  // the estimator's gate decides the error evaluation only in TDB_ERRMODE_MLP; otherwise
  // its decision goes to a scratch word and the host's schedule stands
  const bool mlp = ctx->cfg.error_mode == TDB_ERRMODE_MLP;
  auto features = [&](cudaStream_t q) {
    if (ctx->f64) return;
    int64_t nds = 1;
    for (int n = 0; n < p; ++n) nds *= ctx->r[n];
    est_features(ctx->est_dev, (const float*)ctx->dS, (int)nds, &ctx->rb_dev->dv2, ctx->sig2_lag, ctx->r, p,
                 ctx->mlpP, ctx->mlpNorm, ctx->rb_dev->feat, &ctx->rb_dev->est,
                 mlp ? &ctx->rb_dev->need : ctx->need_scratch, &ctx->rb_dev->ds2, q);
  };
  // a7: error, exact or estimated (the estimator's features and gate first).  Recorded
  // steps enqueue the error kernels on every step, gated by the device word.
  const int* gate = nullptr;
  if (ctx->cfg.error_mode != TDB_ERRMODE_EXACT && (all_paths || ctx->gated_step)) gate = &ctx->rb_dev->need;
  const bool run_error = all_paths || ctx->need_host;
  if (split) {
    CK(cudaEventRecord(ctx->ev_fork, s));
    CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    launch_gram_finish(mode_desc(ctx), ctx->Gpart, gram_split(ctx->r, p, ctx->gsplit), ctx->G, ctx->Ginv, ctx->Ginvf,
                       ctx->sig2, ctx->Vprev, ctx->warm ? 1 : 0, ctx->flags, ctx->aux);
    features(s);
    CHECK_LAUNCH();
    if (run_error) TRY(exact_error2<Tc>(ctx, Vn, gate));
    CK(cudaEventRecord(ctx->ev_join, ctx->aux));
    CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    if (ev) CK(record_timing_event(ev[3], s));
    return readback_enqueue(ctx);
  }
  features(s);
  CHECK_LAUNCH();
  if (run_error) TRY(exact_error2<Tc>(ctx, Vn, gate));
  if (ev) CK(record_timing_event(ev[3], s));
  return readback_enqueue(ctx);
}

// The recorded estimator rows: keep the last tr_cap; compact once the dropped rows number
// tr_cap (amortised O(1) per row).
void trace_trim(tdb_ctx* ctx) {
  const size_t rows = ctx->hT.size();
  if (rows - ctx->tr_off > (size_t)ctx->tr_cap) ctx->tr_off = rows - (size_t)ctx->tr_cap;
  if (ctx->tr_off >= (size_t)ctx->tr_cap) {
    ctx->hX.erase(ctx->hX.begin(), ctx->hX.begin() + ctx->tr_off * MLP_F);
    ctx->hT.erase(ctx->hT.begin(), ctx->hT.begin() + ctx->tr_off);
    ctx->tr_off = 0;
  }
}
int trace_rows(const tdb_ctx* ctx) { return (int)(ctx->hT.size() - ctx->tr_off); }

// After the step record is back: errors, rank control (Sec. 2.5), estimator bookkeeping,
// the step info.
template <typename Tc>
tdb_status finish_step(tdb_ctx* ctx, const Tc* Vn, tdb_step_info* info) {
  const int p = ctx->p;
  ctx->warm = true;
  cudaEvent_t* ev = ctx->prof ? ctx->pev : nullptr;
  float m01 = 0, m12 = 0, m23 = 0, m45 = 0;
  if (ev) {
    cudaError_t e = cudaEventElapsedTime(&m01, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m12, ev[1], ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m23, ev[2], ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m45, ctx->main_from_start ? ev[0] : ev[4], ev[5]);
    if (e != cudaSuccess && ctx->last_graphed) {
      // the events of a recorded step could not be timed: later profiled steps run eagerly
      cudaGetLastError();
      ctx->prof_graph_ok = false;
      ev = nullptr;
    } else {
      CK(e);
    }
  }
  if (ev) {
    ctx->pacc.steps++;
    ctx->pacc.ms_project += m01;
    ctx->pacc.ms_update += m12;
    ctx->pacc.ms_error += m23;
    ctx->pacc.ms_project_main += m45;
    ctx->pacc.launches_main++;
  }
  if (ctx->rb.flags & kFlagNonFinite) { ctx->err = "non-finite value in a snapshot difference"; return TDB_ERR_NONFINITE; }
  if (ctx->rb.flags & kFlagCholGram) { ctx->err = "T_(n) T_(n)^T is not positive definite"; return TDB_ERR_RANK_DEFICIENT; }
  if (ctx->rb.flags & kFlagCholQR) { ctx->err = "U^T W U is not positive definite"; return TDB_ERR_RANK_DEFICIENT; }
  const bool gated = ctx->gated_step;
  const bool exact = gated ? ctx->rb.need != 0 : ctx->need_host;
  const bool feats = !ctx->f64;
  double eps = exact ? std::sqrt(std::max(ctx->rb.err2, 0.0)) : (gated ? ctx->rb.est : NAN);
  double dv2 = ctx->rb.dv2;
  if (exact) ctx->exact_evals++;
  // a8: rank control
  double eps_after = eps;
  int n_re = 0, action = ACT_NONE;
  tdb_status cs = TDB_OK;
  if (exact) {
    auto t0 = std::chrono::steady_clock::now();
    cs = control<Tc>(ctx, Vn, eps, &eps_after, &n_re, &action);
    if (ctx->prof)
      ctx->pacc.ms_control += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (cs != TDB_OK) return cs;
    if (n_re > 0) {
      TRY(readback(ctx));   // sigma of the new state
    }
  }
  // estimator bookkeeping: the trace (features, log10 exact error of the step) and counters
  if (feats) {
    // training row: features and the change of log10 error over this step (target of the network)
    if (exact && eps > 0 && std::isfinite(eps)) {
      ctx->hX.insert(ctx->hX.end(), ctx->rb.feat, ctx->rb.feat + MLP_F);
      ctx->hT.push_back((float)(std::log10(eps) - ctx->est.last_log_eps));
      trace_trim(ctx);
    }
    const double e_now = exact ? eps_after : eps;
    if (e_now > 0 && std::isfinite(e_now)) ctx->est.last_log_eps = std::log10(e_now);
    ctx->est.prev_res_log = ctx->rb.feat[2];
    if (exact) ctx->est.steps_since_exact = 0;
    if (n_re > 0) ctx->est.steps_since_reinit = 0;
  }
  ctx->V_prev2 = ctx->cfg.integrator == TDB_RK2_CENTRAL ? ctx->V_prev : nullptr;
  ctx->V_prev = Vn;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->ds_norm = std::sqrt(std::max(ctx->rb.ds2, 0.0));
    info->eps_est = ctx->est.ready ? ctx->rb.est : NAN;
    info->gate = gated ? ctx->rb.need : 0;
    info->step = ctx->step;
    info->eps = eps_after;
    info->eps_exact = exact ? 1 : 0;
    info->eps_step = eps;
    info->reinit = n_re;
    info->action = action;
    info->dv_norm = std::sqrt(std::max(dv2, 0.0));
    double denom = 0.0;
    for (int n = 0; n < p; ++n) denom += (double)ctx->r[n] * (double)ctx->N[n];
    double rp = 1.0;
    for (int n = 0; n < p; ++n) rp *= ctx->r[n];
    info->cr = (double)ctx->S / (denom + rp);
    for (int n = 0; n < p; ++n) {
      info->ranks[n] = ctx->r[n];
      double tot = 0.0;
      for (int i = 0; i < ctx->r[n]; ++i) tot += std::max(ctx->rb.sig2[n][i], 0.0);
      double e = (eps_after == eps_after) ? eps_after : 0.0;
      info->gamma[n] = tot / (tot + e * e) * 100.0;
      info->sigma_min[n] = std::sqrt(std::max(ctx->rb.sig2[n][ctx->r[n] - 1], 0.0));
    }
  }
  return (action == ACT_CAP) ? TDB_WARN_RANK_CAP : TDB_OK;
}

template <typename Tc>
tdb_status step_impl(tdb_ctx* ctx, const Tc* Vn, tdb_step_info* info) {
  ctx->last_graphed = false;
  prepare_step(ctx);
  TRY(enqueue_step<Tc>(ctx, Vn, (const Tc*)ctx->V_prev, false, (const Tc*)ctx->V_prev2));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(readback_done(ctx));
  return finish_step<Tc>(ctx, Vn, info);
}

// What the recorded step depends on besides data: the ranks and the modes of work.
uint64_t graph_key(const tdb_ctx* ctx) {
  uint64_t k = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { k = (k ^ v) * 1099511628211ull; };
  for (int n = 0; n < ctx->p; ++n) mix((uint64_t)ctx->r[n]);
  mix(ctx->prof ? 1 : 0);
  mix(ctx->warm ? 1 : 0);
  mix((uint64_t)ctx->cfg.error_mode);
  mix(ctx->use_tc ? 1 : 0);
  return k | 1ull;
}

void drop_graphs(tdb_ctx* ctx) {
  for (int i = 0; i < 2; ++i) {
    if (ctx->gexec[i]) cudaGraphExecDestroy(ctx->gexec[i]);
    ctx->gexec[i] = nullptr;
    ctx->gkey[i] = 0;
  }
}


// Record the step with V_{k+1} = Vn, V_k = Vp (and V_{k-1} = Vpp, central differences)
// into an executable graph; count receives the library kernels it holds.
// (The caller's stream may be the legacy default stream, which cannot be captured: the
// work is recorded on a private stream and the graph launched on the caller's.)
template <typename Tc>
tdb_status capture_step(tdb_ctx* ctx, const Tc* Vn, const Tc* Vp, const Tc* Vpp, cudaGraphExec_t* out,
                        long long* count) {
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "capture stream unavailable";
    return TDB_ERR_CUDA;
  }
  cudaStream_t s = ctx->cap_stream;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "stream capture could not begin";
    return TDB_ERR_CUDA;
  }
  cudaStream_t own = ctx->stream;
  ctx->stream = s;
  const long long l0 = launches_so_far();
  tdb_status st = enqueue_step<Tc>(ctx, Vn, Vp, true, Vpp);
  *count = launches_so_far() - l0;
  count_launch(-(int)*count);     // recorded, not launched; counted per replay
  ctx->stream = own;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != TDB_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st == TDB_OK) { ctx->err = std::string("step capture: ") + cudaGetErrorString(e); st = TDB_ERR_CUDA; }
    return st;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(e); return TDB_ERR_CUDA; }
  return TDB_OK;
}

template <typename Tc>
tdb_status step_slot(tdb_ctx* ctx, int parity, tdb_step_info* info) {
  const Tc* Vn = (const Tc*)ctx->slot[parity];
  // the tensor-core plan prepares its constant weights on its first (eager) call.
  // Profiled steps are recorded too: their timing events are external event-record nodes,
  // so the phases are timed as the recorded step runs them (eagerly if the runtime cannot
  // time such events)
  const bool can_graph = !ctx->graph_broken && (!ctx->prof || ctx->prof_graph_ok) && (!ctx->use_tc || ctx->tc.wsl_ready);
  ctx->last_graphed = can_graph;
  if (!can_graph) return step_impl<Tc>(ctx, Vn, info);
  prepare_step(ctx);
  const uint64_t key = graph_key(ctx);
  if (!ctx->gexec[parity] || ctx->gkey[parity] != key) {
    if (ctx->gexec[parity]) cudaGraphExecDestroy(ctx->gexec[parity]);
    ctx->gexec[parity] = nullptr;
    if (capture_step<Tc>(ctx, Vn, (const Tc*)ctx->slot[1 - parity], (const Tc*)nullptr, &ctx->gexec[parity],
                         &ctx->gcount[parity]) != TDB_OK) {
      // stream capture unavailable for this configuration: run this and later steps eagerly
      ctx->graph_broken = true;
      ctx->gexec[parity] = nullptr;
      TRY(enqueue_step<Tc>(ctx, Vn, (const Tc*)ctx->V_prev, false));
      CK(cudaStreamSynchronize(ctx->stream));
      TRY(readback_done(ctx));
      return finish_step<Tc>(ctx, Vn, info);
    }
    ctx->gkey[parity] = key;
    ctx->graph_records++;
  }
  CK(cudaGraphLaunch(ctx->gexec[parity], ctx->stream));
  ctx->graph_replays++;
  count_launch((int)ctx->gcount[parity]);
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(readback_done(ctx));
  return finish_step<Tc>(ctx, Vn, info);
}

// tdb_push_snapshot: a (V_{k+1}, V_k, V_{k-1}) tuple met for the second time is recorded
// (the step's key as for slots, the pointers besides) and replayed while it recurs; the
// least recently used of the kept graphs gives way to a new one.
template <typename Tc>
tdb_status step_pointer(tdb_ctx* ctx, const Tc* Vn, tdb_step_info* info) {
  const void* tup[3] = {Vn, ctx->V_prev, ctx->V_prev2};
  const bool can_graph = !ctx->graph_broken && (!ctx->prof || ctx->prof_graph_ok) && (!ctx->use_tc || ctx->tc.wsl_ready);
  auto same = [&](const void* const* v) { return v[0] == tup[0] && v[1] == tup[1] && v[2] == tup[2]; };
  tdb_ctx::PtrGraph* hit = nullptr;
  if (can_graph)
    for (auto& g : ctx->pgraph)
      if (g.exec && same(g.v)) hit = &g;
  bool seen = false;
  if (can_graph && !hit)
    for (auto& v : ctx->pseen) seen = seen || same(v);
  if (!hit && !seen) {
    if (can_graph) {
      memcpy(ctx->pseen[ctx->pseen_next], tup, sizeof(tup));
      ctx->pseen_next = (ctx->pseen_next + 1) % tdb_ctx::kPtrSeen;
    }
    return step_impl<Tc>(ctx, Vn, info);
  }
  ctx->last_graphed = true;
  prepare_step(ctx);
  const uint64_t key = graph_key(ctx);
  if (!hit) {
    for (auto& g : ctx->pgraph)
      if (!hit && !g.exec) hit = &g;
    if (!hit) {
      hit = &ctx->pgraph[0];
      for (auto& g : ctx->pgraph)
        if (g.used < hit->used) hit = &g;
      cudaGraphExecDestroy(hit->exec);
    }
    *hit = {};
    memcpy(hit->v, tup, sizeof(tup));
  }
  if (!hit->exec || hit->key != key) {
    if (hit->exec) cudaGraphExecDestroy(hit->exec);
    hit->exec = nullptr;
    if (capture_step<Tc>(ctx, Vn, (const Tc*)tup[1], (const Tc*)tup[2], &hit->exec, &hit->count) != TDB_OK) {
      ctx->graph_broken = true;
      *hit = {};
      ctx->last_graphed = false;
      TRY(enqueue_step<Tc>(ctx, Vn, (const Tc*)tup[1], false, (const Tc*)tup[2]));
      CK(cudaStreamSynchronize(ctx->stream));
      TRY(readback_done(ctx));
      return finish_step<Tc>(ctx, Vn, info);
    }
    hit->key = key;
    ctx->graph_records++;
  }
  hit->used = ++ctx->ptick;
  CK(cudaGraphLaunch(hit->exec, ctx->stream));
  ctx->graph_replays++;
  count_launch((int)hit->count);
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(readback_done(ctx));
  return finish_step<Tc>(ctx, Vn, info);
}

tdb_status enqueue_any(tdb_ctx* ctx, int parity) {
  return ctx->f64 ? enqueue_step<double>(ctx, (const double*)ctx->slot[parity], (const double*)ctx->slot[1 - parity], true)
                  : enqueue_step<float>(ctx, (const float*)ctx->slot[parity], (const float*)ctx->slot[1 - parity], true);
}

tdb_status finish_any(tdb_ctx* ctx, int parity, tdb_step_info* info) {
  return ctx->f64 ? finish_step<double>(ctx, (const double*)ctx->slot[parity], info)
                  : finish_step<float>(ctx, (const float*)ctx->slot[parity], info);
}

tdb_status step_any(tdb_ctx* ctx, int parity, tdb_step_info* info) {
  return ctx->f64 ? step_impl<double>(ctx, (const double*)ctx->slot[parity], info)
                  : step_impl<float>(ctx, (const float*)ctx->slot[parity], info);
}

tdb_status slot_check(tdb_ctx* ctx, int parity) {
  if (!ctx->ready) { ctx->err = "push before init"; return TDB_ERR_STATE; }
  if (parity != 0 && parity != 1) { ctx->err = "slot parity must be 0 or 1"; return TDB_ERR_INVALID_ARG; }
  if (!ctx->slot[0] || !ctx->slot[1]) { ctx->err = "input slots not set (tdb_set_input_slots)"; return TDB_ERR_STATE; }
  if (ctx->cfg.integrator == TDB_RK2_CENTRAL) {
    ctx->err = "central differences need three snapshots; use tdb_push_snapshot";
    return TDB_ERR_UNSUPPORTED;
  }
  if (ctx->V_prev != ctx->slot[1 - parity]) {
    ctx->err = "the previous snapshot is not in the other slot";
    return TDB_ERR_STATE;
  }
  return TDB_OK;
}

tdb_status common_init(tdb_ctx** out, const tdb_config* cfg, void* ws, size_t ws_bytes, void* stream, tdb_ctx** made) {
  *made = nullptr;
  if (!out) { g_init_error = "null ctx pointer"; return TDB_ERR_INVALID_ARG; }
  *out = nullptr;
  std::string err;
  tdb_status st = validate(cfg, err);
  if (st != TDB_OK) { g_init_error = err; return st; }
  tdb_ctx* ctx = new (std::nothrow) tdb_ctx();
  if (!ctx) { g_init_error = "out of host memory"; return TDB_ERR_INVALID_ARG; }
  setup_dims(ctx, cfg);
  ctx->stream = (cudaStream_t)stream;
  ctx->use_tc = (ctx->prec == TDB_BF16_TTM);
  if (ctx->use_tc && !tc_supported(ctx->p, ctx->N, ctx->cap, err)) {
    g_init_error = "bf16 tensor-core path: " + err;
    delete ctx;
    return TDB_ERR_UNSUPPORTED;
  }
  Carver size_only(nullptr);
  carve(ctx, size_only);
  size_t need = size_only.off + 256;
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) {
    g_init_error = "workspace null, misaligned or smaller than tdb_workspace_bytes()";
    delete ctx;
    return TDB_ERR_WORKSPACE;
  }
  Carver cv(ws);
  carve(ctx, cv);
  // weights
  for (int n = 0; n < ctx->p; ++n) {
    std::vector<double> wh(ctx->N[n], 1.0);
    if (cfg->weights[n]) {
      for (int64_t i = 0; i < ctx->N[n]; ++i) {
        wh[i] = cfg->weights[n][i];
        if (!(wh[i] > 0.0) || !std::isfinite(wh[i])) {
          g_init_error = "weights must be positive and finite";
          delete ctx;
          return TDB_ERR_INVALID_ARG;
        }
      }
    }
    cudaError_t e = cudaMemcpyAsync(ctx->w[n], wh.data(), sizeof(double) * ctx->N[n], cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      g_init_error = std::string("copying weights: ") + cudaGetErrorString(e);
      delete ctx;
      return TDB_ERR_CUDA;
    }
  }
  if (cudaHostAlloc((void**)&ctx->rb_pin, sizeof(Readback) + sizeof(EstState) + 64, cudaHostAllocDefault) !=
      cudaSuccess) {
    g_init_error = "pinned host memory for the step record unavailable";
    delete ctx;
    return TDB_ERR_CUDA;
  }
  // the second branch of exact-error steps (without it those steps run on one stream)
  if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    ctx->aux = nullptr;
    ctx->ev_fork = ctx->ev_join = nullptr;
  }
  ctx->est_pin = (EstState*)((char*)ctx->rb_pin + ((sizeof(Readback) + 15) & ~(size_t)15));
  ctx->need_pin = (int*)((char*)ctx->est_pin + ((sizeof(EstState) + 15) & ~(size_t)15));
  {
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, ctx->rb_pin, 0) == cudaSuccess && dp) {
      char* base = (char*)dp;
      ctx->est_pin_d = (const EstState*)(base + ((char*)ctx->est_pin - (char*)ctx->rb_pin));
      ctx->need_pin_d = (const int*)(base + ((char*)ctx->need_pin - (char*)ctx->rb_pin));
    } else {
      cudaGetLastError();
    }
  }
  cudaMemsetAsync(ctx->rb_dev, 0, sizeof(Readback), ctx->stream);
  cudaMemsetAsync(ctx->redcnt, 0, 8 * sizeof(unsigned), ctx->stream);
  if (ctx->f64)
    launch_weights_T<double>(weight_view(ctx), (double*)ctx->w1T, (double*)ctx->wcolT, ctx->stream);
  else
    launch_weights_T<float>(weight_view(ctx), (float*)ctx->w1T, (float*)ctx->wcolT, ctx->stream);
  memset(&ctx->est, 0, sizeof(ctx->est));
  ctx->est.last_log_eps = -30.0;
  ctx->est.max_skip = std::max(1, ctx->cfg.error_every);
  ctx->est.gate = 0.5;
  ctx->est.eps_th = ctx->cfg.eps_th;
  ctx->est.novelty_z = 8.0;
  ctx->est.prev_res_log = -30.0;
  if (ctx->cfg.error_mode == TDB_ERRMODE_MLP && ctx->f64) {
    g_init_error = "the learned estimator runs in the FP32 and BF16 modes";
    delete ctx;
    return TDB_ERR_UNSUPPORTED;
  }
  *made = ctx;
  return TDB_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

size_t tdb_workspace_bytes(const tdb_config* cfg) {
  std::string err;
  if (validate(cfg, err) != TDB_OK) return 0;
  tdb_ctx c;
  setup_dims(&c, cfg);
  Carver cv(nullptr);
  carve(&c, cv);
  return cv.off + 256;
}

tdb_status tdb_init(tdb_ctx** out, const tdb_config* cfg, void* ws, size_t ws_bytes, const void* V0, void* stream) {
  tdb_ctx* ctx = nullptr;
  tdb_status st = common_init(out, cfg, ws, ws_bytes, stream, &ctx);
  if (st != TDB_OK) return st;
  if (!V0) { g_init_error = "null V0"; delete ctx; return TDB_ERR_INVALID_ARG; }
  auto run = [&](auto tag) -> tdb_status {
    using Tc = decltype(tag);
    const Tc* V = (const Tc*)V0;
    TRY(hosvd_spectrum<Tc>(ctx, V));
    std::vector<int> r(ctx->p);
    for (int n = 0; n < ctx->p; ++n) {
      if (cfg->rank[n] > 0)
        r[n] = std::min(cfg->rank[n], ctx->cap[n]);
      else
        r[n] = std::min(ctx->cap[n], rank_from_spectrum(ctx->h_ev[n], ctx->h_trace[n], cfg->gamma_th));
    }
    r = clamp_product_bound(r);
    TRY(hosvd_state<Tc>(ctx, V, r.data()));
    TRY(readback(ctx));
    if (!ctx->f64) TRY(seed_estimator<Tc>(ctx, V));
    return TDB_OK;
  };
  st = ctx->f64 ? run(double()) : run(float());
  if (st != TDB_OK) {
    g_init_error = ctx->err;
    delete ctx;
    return st;
  }
  ctx->V_prev = V0;
  ctx->V_prev2 = nullptr;
  ctx->ready = true;
  *out = ctx;
  return TDB_OK;
}

tdb_status tdb_init_from_factors(tdb_ctx** out, const tdb_config* cfg, void* ws, size_t ws_bytes, const double* core,
                                 const double* const* U, const int* ranks, const void* V0, void* stream) {
  tdb_ctx* ctx = nullptr;
  tdb_status st = common_init(out, cfg, ws, ws_bytes, stream, &ctx);
  if (st != TDB_OK) return st;
  if (!V0 || !core || !U || !ranks) { g_init_error = "null argument"; delete ctx; return TDB_ERR_INVALID_ARG; }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) {
    int other = 1;
    for (int m = 0; m < ctx->p; ++m)
      if (m != n) other *= ranks[m];
    if (ranks[n] < 1 || ranks[n] > ctx->cap[n] || ranks[n] > other || !U[n]) {
      g_init_error = "rank outside 1..min(N_n, prod_{m!=n} r_m, rank cap)";
      delete ctx;
      return TDB_ERR_RANK;
    }
    ctx->r[n] = ranks[n];
    Rprod *= ranks[n];
  }
  cudaError_t e = cudaMemcpyAsync(ctx->T, core, sizeof(double) * Rprod, cudaMemcpyHostToDevice, ctx->stream);
  for (int n = 0; n < ctx->p && e == cudaSuccess; ++n)
    e = cudaMemcpyAsync(ctx->U[n], U[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    g_init_error = std::string("copying factors: ") + cudaGetErrorString(e);
    delete ctx;
    return TDB_ERR_CUDA;
  }
  st = ctx->f64 ? refresh_derived<double>(ctx, true) : refresh_derived<float>(ctx, true);
  if (st == TDB_OK) st = readback(ctx);
  if (st == TDB_OK && !ctx->f64) st = seed_estimator<float>(ctx, (const float*)V0);
  if (st != TDB_OK) {
    g_init_error = ctx->err;
    delete ctx;
    return st;
  }
  ctx->V_prev = V0;
  ctx->V_prev2 = nullptr;
  ctx->ready = true;
  *out = ctx;
  return TDB_OK;
}

tdb_status tdb_push_snapshot(tdb_ctx* ctx, const void* V_next, tdb_step_info* info) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "push before init"; return TDB_ERR_STATE; }
  if (!V_next) { ctx->err = "null snapshot"; return TDB_ERR_INVALID_ARG; }
  ctx->last_graphed = false;
  return ctx->f64 ? step_pointer<double>(ctx, (const double*)V_next, info)
                  : step_pointer<float>(ctx, (const float*)V_next, info);
}

tdb_status tdb_reconstruct(tdb_ctx* ctx, void* V_out) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "reconstruct before init"; return TDB_ERR_STATE; }
  if (!V_out) { ctx->err = "null output"; return TDB_ERR_INVALID_ARG; }
  return ctx->f64 ? reconstruct_into<double>(ctx, (double*)V_out) : reconstruct_into<float>(ctx, (float*)V_out);
}

tdb_status tdb_adapt_rank(tdb_ctx* ctx, const void* V_now, int* ranks_out, double* eps_out) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "adapt before init"; return TDB_ERR_STATE; }
  if (!V_now) { ctx->err = "null snapshot"; return TDB_ERR_INVALID_ARG; }
  auto run = [&](auto tag) -> tdb_status {
    using Tc = decltype(tag);
    double eps, ea;
    int nre, act;
    TRY(error_now<Tc>(ctx, (const Tc*)V_now, &eps));
    TRY(control<Tc>(ctx, (const Tc*)V_now, eps, &ea, &nre, &act));
    if (eps_out) *eps_out = ea;
    return act == ACT_CAP ? TDB_WARN_RANK_CAP : TDB_OK;
  };
  tdb_status st = ctx->f64 ? run(double()) : run(float());
  // the state now stands for V_now (re-initialised from it, or accepted against it):
  // the next push differences against V_now
  if (st == TDB_OK || st == TDB_WARN_RANK_CAP) {
    ctx->V_prev = V_now;
    ctx->V_prev2 = nullptr;
  }
  if (ranks_out)
    for (int n = 0; n < ctx->p; ++n) ranks_out[n] = ctx->r[n];
  return st;
}

tdb_status tdb_reinit(tdb_ctx* ctx, const void* V_now) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "reinit before init"; return TDB_ERR_STATE; }
  if (!V_now) { ctx->err = "null snapshot"; return TDB_ERR_INVALID_ARG; }
  auto run = [&](auto tag) -> tdb_status {
    using Tc = decltype(tag);
    const Tc* V = (const Tc*)V_now;
    std::vector<int> r(ctx->r, ctx->r + ctx->p);
    TRY(hosvd_spectrum<Tc>(ctx, V));
    TRY(hosvd_state<Tc>(ctx, V, r.data()));
    return readback(ctx);
  };
  const tdb_status st = ctx->f64 ? run(double()) : run(float());
  if (st == TDB_OK) {
    ctx->history.clear();
    ctx->reinits += 1;
    ctx->V_prev = V_now;
    ctx->V_prev2 = nullptr;
  }
  return st;
}

tdb_status tdb_get_factors(tdb_ctx* ctx, double* core, double* const* U, int* ranks) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "not initialised"; return TDB_ERR_STATE; }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) Rprod *= ctx->r[n];
  if (core) CK(cudaMemcpyAsync(core, ctx->T, sizeof(double) * Rprod, cudaMemcpyDeviceToHost, ctx->stream));
  if (U)
    for (int n = 0; n < ctx->p; ++n)
      if (U[n]) CK(cudaMemcpyAsync(U[n], ctx->U[n], sizeof(double) * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ranks)
    for (int n = 0; n < ctx->p; ++n) ranks[n] = ctx->r[n];
  return TDB_OK;
}

tdb_status tdb_get_projection(tdb_ctx* ctx, double* dS, double* const* Y) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "not initialised"; return TDB_ERR_STATE; }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) Rprod *= ctx->r[n];
  auto fetch = [&](const void* src, double* dst, int64_t cnt) -> tdb_status {
    if (ctx->f64) {
      CK(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    } else {
      std::vector<float> tmp(cnt);
      CK(cudaMemcpyAsync(tmp.data(), src, sizeof(float) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int64_t i = 0; i < cnt; ++i) dst[i] = tmp[i];
    }
    return TDB_OK;
  };
  if (dS) TRY(fetch(ctx->dS, dS, Rprod));
  if (Y)
    for (int n = 0; n < ctx->p; ++n)
      if (Y[n]) TRY(fetch(ctx->Y[n], Y[n], Rprod / ctx->r[n] * ctx->N[n]));
  return TDB_OK;
}

tdb_status tdb_get_counters(tdb_ctx* ctx, int64_t* steps, int64_t* reinits, int64_t* exact_evals) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (steps) *steps = ctx->step;
  if (reinits) *reinits = ctx->reinits;
  if (exact_evals) *exact_evals = ctx->exact_evals;
  return TDB_OK;
}

// Serialised layout: magic, p, ranks[4], step, reinits, exact_evals, nhist, history[nhist], T, U_n.
tdb_status tdb_save_state(tdb_ctx* ctx, void* buf, size_t* bytes) {
  if (!ctx || !bytes) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready) { ctx->err = "not initialised"; return TDB_ERR_STATE; }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) Rprod *= ctx->r[n];
  size_t need = 8 * (1 + 1 + kMaxModes + 3 + 1) + 8 * ctx->history.size() + 8 * Rprod;
  for (int n = 0; n < ctx->p; ++n) need += 8 * ctx->N[n] * ctx->r[n];
  if (!buf) { *bytes = need; return TDB_OK; }
  if (*bytes < need) { *bytes = need; ctx->err = "buffer too small"; return TDB_ERR_INVALID_ARG; }
  int64_t* h = (int64_t*)buf;
  h[0] = 0x54444231;  // "TDB1"
  h[1] = ctx->p;
  for (int n = 0; n < kMaxModes; ++n) h[2 + n] = n < ctx->p ? ctx->r[n] : 0;
  h[6] = ctx->step;
  h[7] = ctx->reinits;
  h[8] = ctx->exact_evals;
  h[9] = (int64_t)ctx->history.size();
  double* d = (double*)(h + 10);
  for (size_t i = 0; i < ctx->history.size(); ++i) d[i] = ctx->history[i];
  d += ctx->history.size();
  CK(cudaMemcpyAsync(d, ctx->T, 8 * Rprod, cudaMemcpyDeviceToHost, ctx->stream));
  d += Rprod;
  for (int n = 0; n < ctx->p; ++n) {
    CK(cudaMemcpyAsync(d, ctx->U[n], 8 * ctx->N[n] * ctx->r[n], cudaMemcpyDeviceToHost, ctx->stream));
    d += ctx->N[n] * ctx->r[n];
  }
  CK(cudaStreamSynchronize(ctx->stream));
  *bytes = need;
  return TDB_OK;
}

tdb_status tdb_load_state(tdb_ctx* ctx, const void* buf, size_t bytes, const void* V_prev) {
  if (!ctx || !buf || !V_prev) return TDB_ERR_INVALID_ARG;
  const int64_t* h = (const int64_t*)buf;
  if (bytes < 80 || h[0] != 0x54444231 || h[1] != ctx->p) { ctx->err = "not a state of this configuration"; return TDB_ERR_INVALID_ARG; }
  int64_t Rprod = 1;
  for (int n = 0; n < ctx->p; ++n) {
    if (h[2 + n] < 1 || h[2 + n] > ctx->cap[n]) { ctx->err = "saved rank exceeds this context's cap"; return TDB_ERR_RANK; }
    ctx->r[n] = (int)h[2 + n];
    Rprod *= ctx->r[n];
  }
  ctx->step = h[6];
  ctx->reinits = h[7];
  ctx->exact_evals = h[8];
  int64_t nh = h[9];
  size_t need = 80 + 8 * (size_t)nh + 8 * Rprod;
  for (int n = 0; n < ctx->p; ++n) need += 8 * ctx->N[n] * ctx->r[n];
  if (bytes < need) { ctx->err = "state buffer truncated"; return TDB_ERR_INVALID_ARG; }
  const double* d = (const double*)(h + 10);
  ctx->history.assign(d, d + nh);
  d += nh;
  CK(cudaMemcpyAsync(ctx->T, d, 8 * Rprod, cudaMemcpyHostToDevice, ctx->stream));
  d += Rprod;
  for (int n = 0; n < ctx->p; ++n) {
    CK(cudaMemcpyAsync(ctx->U[n], d, 8 * ctx->N[n] * ctx->r[n], cudaMemcpyHostToDevice, ctx->stream));
    d += ctx->N[n] * ctx->r[n];
  }
  ctx->warm = false;
  tdb_status st = ctx->f64 ? refresh_derived<double>(ctx, true) : refresh_derived<float>(ctx, true);
  if (st != TDB_OK) return st;
  TRY(readback(ctx));
  ctx->V_prev = V_prev;
  ctx->V_prev2 = nullptr;
  ctx->ready = true;
  return TDB_OK;
}

const char* tdb_last_error(const tdb_ctx* ctx) {
  if (!ctx) return g_init_error.c_str();
  return ctx->err.c_str();
}

const char* tdb_status_string(tdb_status s) {
  switch (s) {
    case TDB_OK: return "TDB_OK";
    case TDB_ERR_INVALID_ARG: return "TDB_ERR_INVALID_ARG";
    case TDB_ERR_SHAPE: return "TDB_ERR_SHAPE";
    case TDB_ERR_RANK: return "TDB_ERR_RANK";
    case TDB_ERR_RANK_DEFICIENT: return "TDB_ERR_RANK_DEFICIENT";
    case TDB_ERR_NONFINITE: return "TDB_ERR_NONFINITE";
    case TDB_ERR_CUDA: return "TDB_ERR_CUDA";
    case TDB_ERR_TIMEOUT: return "TDB_ERR_TIMEOUT";
    case TDB_ERR_STATE: return "TDB_ERR_STATE";
    case TDB_WARN_RANK_CAP: return "TDB_WARN_RANK_CAP";
    case TDB_ERR_WORKSPACE: return "TDB_ERR_WORKSPACE";
    case TDB_ERR_UNSUPPORTED: return "TDB_ERR_UNSUPPORTED";
  }
  return "unknown status";
}

tdb_status tdb_estimator_fit(tdb_ctx* ctx, int iters, float lr, uint64_t seed, double gate, double* loss_out) {
  if (!ctx || iters < 1 || !(lr > 0) || !(gate > 0)) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready || ctx->f64) { ctx->err = "estimator needs an initialised FP32/BF16 context"; return TDB_ERR_STATE; }
  const int n = trace_rows(ctx);
  if (n < 16) { ctx->err = "fewer than 16 exact evaluations recorded"; return TDB_ERR_STATE; }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(ctx->trX, ctx->hX.data() + ctx->tr_off * MLP_F, sizeof(float) * n * MLP_F,
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->trT, ctx->hT.data() + ctx->tr_off, sizeof(float) * n, cudaMemcpyHostToDevice, s));
  est_normalize(ctx->trX, ctx->trT, n, ctx->mlpNorm, s);
  est_init_params(ctx->mlpP, (unsigned long long)seed, s);
  CK(cudaMemsetAsync(ctx->mlpM, 0, sizeof(float) * MLP_NPARAM, s));
  CK(cudaMemsetAsync(ctx->mlpV, 0, sizeof(float) * MLP_NPARAM, s));
  for (int it = 1; it <= iters; ++it) {
    mlp_loss_grad(ctx->mlpP, ctx->trX, ctx->trT, n, ctx->mlpGpart, ctx->mlpLpart, ctx->mlp_parts, ctx->mlpG,
                  ctx->mlpLoss, s);
    mlp_adam(ctx->mlpP, ctx->mlpG, ctx->mlpM, ctx->mlpV, it, lr, s);
  }
  CHECK_LAUNCH();
  float loss = 0.f;
  CK(cudaMemcpyAsync(&loss, ctx->mlpLoss, sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (loss_out) *loss_out = loss;
  ctx->est.ready = 1;
  ctx->est.gate = gate;
  return TDB_OK;
}

tdb_status tdb_estimator_params(tdb_ctx* ctx, float* get_out, const float* set_in, double gate) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->ready || ctx->f64) { ctx->err = "estimator needs an initialised FP32/BF16 context"; return TDB_ERR_STATE; }
  cudaStream_t s = ctx->stream;
  if (get_out) {
    CK(cudaMemcpyAsync(get_out, ctx->mlpP, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(get_out + MLP_NPARAM, ctx->mlpNorm, sizeof(float) * (2 * MLP_F + 2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (set_in) {
    CK(cudaMemcpyAsync(ctx->mlpP, set_in, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->mlpNorm, set_in + MLP_NPARAM, sizeof(float) * (2 * MLP_F + 2), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    ctx->est.ready = 1;
    if (gate > 0) ctx->est.gate = gate;
  }
  return TDB_OK;
}

tdb_status tdb_estimator_trace(tdb_ctx* ctx, float* X, float* t, int* n) {
  if (!ctx || !n) return TDB_ERR_INVALID_ARG;
  const int have = trace_rows(ctx);
  if (X && t) {
    const int m = std::min(*n, have);
    memcpy(X, ctx->hX.data() + ctx->tr_off * MLP_F, sizeof(float) * m * MLP_F);
    memcpy(t, ctx->hT.data() + ctx->tr_off, sizeof(float) * m);
  }
  *n = have;
  return TDB_OK;
}

tdb_status tdb_estimator_load_trace(tdb_ctx* ctx, const float* X, const float* t, int n, int append) {
  if (!ctx || !X || !t || n < 1) return TDB_ERR_INVALID_ARG;
  if (!append) {
    ctx->hX.clear();
    ctx->hT.clear();
    ctx->tr_off = 0;
  }
  ctx->hX.insert(ctx->hX.end(), X, X + (size_t)n * MLP_F);
  ctx->hT.insert(ctx->hT.end(), t, t + n);
  trace_trim(ctx);
  return TDB_OK;
}

tdb_status tdb_set_profiling(tdb_ctx* ctx, int enable) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (enable) {
    for (int i = 0; i < 6; ++i)
      if (!ctx->pev[i]) CK(cudaEventCreate(&ctx->pev[i]));
    memset(&ctx->pacc, 0, sizeof(ctx->pacc));
    CK(cudaMemsetAsync(ctx->stamps, 0, 32 * sizeof(unsigned long long), ctx->stream));
    static const unsigned long long span0[4] = {~0ull, 0ull, 0ull, 0ull};
    CK(cudaMemcpyAsync(ctx->span_dev, span0, sizeof(span0), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  ctx->prof = enable != 0;
  return TDB_OK;
}

tdb_status tdb_get_profile(tdb_ctx* ctx, tdb_profile* out) {
  if (!ctx || !out) return TDB_ERR_INVALID_ARG;
  unsigned long long st[32];
  CK(cudaMemcpyAsync(st, ctx->stamps, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long sp[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(sp, ctx->span_dev, sizeof(sp), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->pacc.us_project_span = 1e-3 * (double)sp[2];
  ctx->pacc.spans = (int64_t)sp[3];
  ctx->pacc.update_phases = std::min(6 + ctx->p, 12);
  for (int k = 0; k < 12; ++k) ctx->pacc.us_update_phase[k] = k < ctx->pacc.update_phases ? 1e-3 * (double)st[16 + k] : 0.0;
  *out = ctx->pacc;
  return TDB_OK;
}

int64_t tdb_kernel_launches(void) { return (int64_t)tdb::launches_so_far(); }

void tdb_destroy(tdb_ctx* ctx) {
  if (!ctx) return;
  for (int i = 0; i < 6; ++i)
    if (ctx->pev[i]) cudaEventDestroy(ctx->pev[i]);
  delete ctx;
}

tdb_status tdb_set_input_slots(tdb_ctx* ctx, const void* slot0, const void* slot1) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if ((slot0 == nullptr) != (slot1 == nullptr) || (slot0 && slot0 == slot1)) {
    ctx->err = "two distinct slots, or none";
    return TDB_ERR_INVALID_ARG;
  }
  ctx->slot[0] = slot0;
  ctx->slot[1] = slot1;
  drop_graphs(ctx);
  return TDB_OK;
}

tdb_status tdb_push_slot(tdb_ctx* ctx, int parity, tdb_step_info* info) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  TRY(slot_check(ctx, parity));
  return ctx->f64 ? step_slot<double>(ctx, parity, info) : step_slot<float>(ctx, parity, info);
}

tdb_status tdb_batch_create(tdb_batch** out, tdb_ctx* const* members, int n, int nstreams, void* stream) {
  if (!out || !members || n < 1 || nstreams < 1) return TDB_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!members[i] || !members[i]->ready) return TDB_ERR_STATE;
    if (members[i]->cfg.integrator == TDB_RK2_CENTRAL) return TDB_ERR_UNSUPPORTED;   // slots hold two snapshots
  }
  tdb_batch* b = new (std::nothrow) tdb_batch();
  if (!b) return TDB_ERR_INVALID_ARG;
  b->m.assign(members, members + n);
  b->main = (cudaStream_t)stream;
  const int ns = std::min(nstreams, n);
  for (int k = 0; k < ns; ++k) {
    cudaStream_t q = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      if (q) cudaStreamDestroy(q);
      delete b;
      return TDB_ERR_CUDA;
    }
    b->st.push_back(q);
    b->join.push_back(e);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return TDB_ERR_CUDA;
  }
  *out = b;
  return TDB_OK;
}

// Record every member's step, member i on stream i mod nstreams, into one graph.
static tdb_status batch_capture(tdb_batch* b, int parity) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    b->err = "batch capture could not begin";
    return TDB_ERR_CUDA;
  }
  tdb_status st = TDB_OK;
  const long long l0 = launches_so_far();
  cudaEventRecord(b->fork, b->cap);
  for (size_t k = 0; k < b->st.size(); ++k) cudaStreamWaitEvent(b->st[k], b->fork, 0);
  for (size_t i = 0; i < b->m.size() && st == TDB_OK; ++i) {
    tdb_ctx* c = b->m[i];
    cudaStream_t own = c->stream;
    c->stream = b->st[i % b->st.size()];
    st = enqueue_any(c, parity);
    c->stream = own;
    if (st != TDB_OK) b->err = "member " + std::to_string(i) + ": " + c->err;
  }
  for (size_t k = 0; k < b->st.size(); ++k) {
    cudaEventRecord(b->join[k], b->st[k]);
    cudaStreamWaitEvent(b->cap, b->join[k], 0);
  }
  b->gcount[parity] = launches_so_far() - l0;
  count_launch(-(int)b->gcount[parity]);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != TDB_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st == TDB_OK) { b->err = std::string("batch capture: ") + cudaGetErrorString(e); st = TDB_ERR_CUDA; }
    return st;
  }
  e = cudaGraphInstantiate(&b->gexec[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { b->err = std::string("batch instantiate: ") + cudaGetErrorString(e); return TDB_ERR_CUDA; }
  return TDB_OK;
}

tdb_status tdb_batch_push(tdb_batch* b, int parity, tdb_step_info* infos) {
  if (!b) return TDB_ERR_INVALID_ARG;
  const size_t n = b->m.size();
  bool eager = b->broken;
  for (size_t i = 0; i < n; ++i) {
    tdb_ctx* c = b->m[i];
    tdb_status st = slot_check(c, parity);
    if (st != TDB_OK) { b->err = "member " + std::to_string(i) + ": " + c->err; return st; }
    if ((c->use_tc && !c->tc.wsl_ready) || c->prof) eager = true;
  }
  tdb_status worst = TDB_OK;
  auto note = [&](tdb_status st, size_t i) {
    if (st == TDB_OK) return;
    if (worst == TDB_OK || (worst == TDB_WARN_RANK_CAP && st != TDB_WARN_RANK_CAP)) {
      worst = st;
      b->err = "member " + std::to_string(i) + ": " + b->m[i]->err;
    }
  };
  if (eager) {
    for (size_t i = 0; i < n; ++i) note(step_any(b->m[i], parity, infos ? infos + i : nullptr), i);
    return worst;
  }
  for (size_t i = 0; i < n; ++i) prepare_step(b->m[i]);
  bool fresh = b->gexec[parity] != nullptr && b->keys[parity].size() == n;
  for (size_t i = 0; i < n && fresh; ++i) fresh = b->keys[parity][i] == graph_key(b->m[i]);
  if (!fresh) {
    if (b->gexec[parity]) cudaGraphExecDestroy(b->gexec[parity]);
    b->gexec[parity] = nullptr;
    if (batch_capture(b, parity) != TDB_OK) {
      // capture unavailable: this and later steps run member by member
      b->broken = true;
      b->gexec[parity] = nullptr;
      for (size_t i = 0; i < n; ++i) {
        tdb_ctx* c = b->m[i];
        c->last_graphed = false;
        tdb_status st = enqueue_any(c, parity);
        if (st == TDB_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = TDB_ERR_CUDA;
        if (st == TDB_OK) st = readback_done(c);
        if (st == TDB_OK) st = finish_any(c, parity, infos ? infos + i : nullptr);
        note(st, i);
      }
      return worst;
    }
    b->keys[parity].resize(n);
    for (size_t i = 0; i < n; ++i) b->keys[parity][i] = graph_key(b->m[i]);
    b->records++;
  }
  b->replays++;
  if (cudaGraphLaunch(b->gexec[parity], b->main) != cudaSuccess || cudaStreamSynchronize(b->main) != cudaSuccess) {
    b->err = std::string("batch graph: ") + cudaGetErrorString(cudaGetLastError());
    return TDB_ERR_CUDA;
  }
  count_launch((int)b->gcount[parity]);
  for (size_t i = 0; i < n; ++i) {
    tdb_ctx* c = b->m[i];
    c->last_graphed = true;
    tdb_status st = readback_done(c);
    if (st == TDB_OK) st = finish_any(c, parity, infos ? infos + i : nullptr);
    note(st, i);
  }
  return worst;
}

const char* tdb_batch_last_error(const tdb_batch* b) { return b ? b->err.c_str() : "null batch"; }

tdb_status tdb_get_graph_counters(const tdb_ctx* ctx, const tdb_batch* b, int64_t* replays, int64_t* records) {
  if ((ctx == nullptr) == (b == nullptr)) return TDB_ERR_INVALID_ARG;
  if (replays) *replays = ctx ? ctx->graph_replays : b->replays;
  if (records) *records = ctx ? ctx->graph_records : b->records;
  return TDB_OK;
}

void tdb_batch_destroy(tdb_batch* b) { delete b; }

tdb_status tdb_tc_tuning(const tdb_ctx* ctx, int* ctas, int* fin_target, int* ncand, int* cand, float* cand_us,
                         int* fin_cand, float* fin_us) {
  if (!ctx) return TDB_ERR_INVALID_ARG;
  if (!ctx->use_tc || !ctx->tc.tuned) return TDB_ERR_STATE;
  const TcPlan& t = ctx->tc;
  if (ctas) *ctas = t.cstep;
  if (fin_target) *fin_target = t.fin_target;
  if (ncand) *ncand = t.ncand;
  for (int i = 0; i < t.ncand; ++i) {
    if (cand) cand[i] = t.cand[i];
    if (cand_us) cand_us[i] = t.cand_us[i];
  }
  for (int i = 0; i < 3; ++i) {
    if (fin_cand) fin_cand[i] = t.ncand ? t.fin_cand[i] : 0;
    if (fin_us) fin_us[i] = t.ncand ? t.fin_us[i] : 0.f;
  }
  return TDB_OK;
}

const char* tdb_version(void) { return "tdb 0.3 sm_103a"; }

}  // extern "C"
