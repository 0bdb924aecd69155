// Host side of libxk: the C ABI of include/xk.h.  Handles own the
// per-geometry tables and the build scratch in device memory; builds are
// sequences of kernel launches on the handle's stream; submissions ride
// pinned host slots and CUDA events so that builds of different handles
// overlap on the GPU.
#include "xk_internal.h"
#include "xk_mixed.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <deque>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "xk.h"

namespace {

thread_local std::string t_err;

int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(XK_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define XK_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

constexpr int kSlots = 4;

struct Slot {
  double* C = nullptr;    // pinned, N x n
  double* K = nullptr;    // pinned, N x n
  double* Ex = nullptr;   // pinned, 1
  int* st = nullptr;      // pinned, 4: the status word of this slot's build
  cudaEvent_t done = nullptr;
  int state = 0;          // 0 free, 1 in flight, 2 abandoned (timed out)
  xk_ticket ticket = 0;
  std::chrono::steady_clock::time_point deadline;
  bool has_deadline = false;
};

// Set-ups in progress (any thread): while one runs, a handle does not capture
// its build graph (capture and instantiation wait behind the set-up's large
// host-to-device copies and stalled that build by up to seconds).
std::atomic<int> g_setups_running{0};
struct SetupMark {
  SetupMark() { g_setups_running.fetch_add(1); }
  ~SetupMark() { g_setups_running.fetch_sub(1); }
};

size_t g_admitted = 0;    // bytes held by live handles and reservations (all devices)
std::mutex g_admit_mu;

// Queued admission: a request that does not fit waits, in arrival order,
// until the bytes it needs are free; releasing a handle or a reservation
// wakes the waiters.  Reservations (xk_admit_reserve) are host bookkeeping
// only: they count against the budget until released.
std::condition_variable g_admit_cv;
std::deque<uint64_t> g_admit_queue;                   // waiting requests, oldest first
uint64_t g_admit_seq = 0;                             // ids of requests and reservation tokens
std::unordered_map<uint64_t, size_t> g_reservations;  // token -> bytes
size_t g_reserved = 0;                                // bytes of live reservations

// Bytes the budget admits now (g_admit_mu held): XK_HBM_BUDGET_BYTES less
// everything admitted, checked first and without any device call; then, if
// `device`, the current device's free memory less 1 GiB and less the
// reservations (which hold no device memory of their own).
int admit_left(bool device, size_t* left, bool* env_short) {
  *left = SIZE_MAX;
  *env_short = false;
  if (const char* env = std::getenv("XK_HBM_BUDGET_BYTES")) {
    const size_t cap = (size_t)std::strtoull(env, nullptr, 10);
    *left = cap > g_admitted ? cap - g_admitted : 0;
    *env_short = true;
  }
  if (device) {
    size_t freeb = 0, totalb = 0;
    cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    const size_t reserve = (size_t)1 << 30;
    size_t dev = freeb > reserve ? freeb - reserve : 0;
    dev = dev > g_reserved ? dev - g_reserved : 0;
    if (dev < *left) {
      *left = dev;
      *env_short = false;
    }
  }
  return XK_OK;
}

// Admits `bytes` (adds them to g_admitted) or fails.  timeout_ms < 0: now or
// XK_ENOMEM.  Otherwise the request queues behind earlier ones and waits up to
// timeout_ms for the bytes (re-checking the device every 50 ms, since other
// processes free memory without waking us): XK_ETIMEDOUT when the wait runs
// out.  A request above XK_HBM_BUDGET_BYTES itself fails at once.
int admit_bytes(size_t bytes, double timeout_ms, bool device, const char* who) {
  std::unique_lock<std::mutex> lk(g_admit_mu);
  if (const char* env = std::getenv("XK_HBM_BUDGET_BYTES")) {
    const size_t cap = (size_t)std::strtoull(env, nullptr, 10);
    if (bytes > cap)
      return fail(XK_ENOMEM, std::string(who) + ": footprint " + std::to_string(bytes) +
                                 " bytes exceeds XK_HBM_BUDGET_BYTES (" + std::to_string(cap) +
                                 " bytes)");
  }
  size_t left = 0;
  bool env_short = false;
  if (timeout_ms < 0.0) {
    // the caller's budget first, before any device call
    int rc = admit_left(false, &left, &env_short);
    if (rc == XK_OK && bytes > left)
      return fail(XK_ENOMEM, std::string(who) + ": footprint " + std::to_string(bytes) +
                                 " bytes exceeds XK_HBM_BUDGET_BYTES less the live handles (" +
                                 std::to_string(left) + " bytes)");
    rc = admit_left(device, &left, &env_short);
    if (rc != XK_OK) return rc;
    if (bytes > left)
      return fail(XK_ENOMEM, std::string(who) + ": footprint " + std::to_string(bytes) +
                                 " bytes exceeds the admission budget " + std::to_string(left));
    g_admitted += bytes;
    return XK_OK;
  }
  const uint64_t id = ++g_admit_seq;
  g_admit_queue.push_back(id);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds((long long)(timeout_ms * 1000.0));
  auto leave = [&]() {
    for (auto it = g_admit_queue.begin(); it != g_admit_queue.end(); ++it)
      if (*it == id) { g_admit_queue.erase(it); break; }
    g_admit_cv.notify_all();
  };
  for (;;) {
    if (g_admit_queue.front() == id) {
      int rc = admit_left(false, &left, &env_short);
      if (rc == XK_OK && bytes <= left) rc = admit_left(device, &left, &env_short);
      if (rc != XK_OK) { leave(); return rc; }
      if (bytes <= left) {
        g_admit_queue.pop_front();
        g_admitted += bytes;
        g_admit_cv.notify_all();  // the next in line may fit too
        return XK_OK;
      }
    }
    const auto now = std::chrono::steady_clock::now();
    if (now >= deadline) {
      leave();
      return fail(XK_ETIMEDOUT, std::string(who) + ": " + std::to_string(bytes) +
                                    " bytes not admitted within the timeout");
    }
    g_admit_cv.wait_for(lk, std::min<std::chrono::steady_clock::duration>(
                                deadline - now, std::chrono::milliseconds(50)));
  }
}

// Returns bytes to the budget and wakes the waiters.
void unadmit_bytes(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_admit_mu);
  g_admitted -= std::min(g_admitted, bytes);
  g_admit_cv.notify_all();
}

}  // namespace

struct xk_handle {
  int64_t Ng = 0;
  int N = 0, n = 0, Naux = 0, mode = 0, device = 0;
  // The handle holds the rows of V and W of the interpolation points
  // [g0, g0 + ga) (all Naux points unless it is a shard) and returns that
  // slice's share of K_{mu i} and E_x; the orbitals are gathered at all Naux.
  int g0 = 0, ga = 0;
  double dV = 0.0;
  size_t footprint = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  bool has_build = false;
  std::vector<void*> allocs;

  // FP64 tables and scratch
  double *phi = nullptr, *phig = nullptr, *V = nullptr, *W = nullptr;
  int32_t* idx = nullptr;
  double* Ce = nullptr;  // xk_energy: C (N x n) and E_x (one more double), apart from the build's
  // xk_build_full: K_{mu nu} (N x N); FP64 path also M_A, M_C (N_aux x N), Y, Z (N x N)
  double *Kf = nullptr, *MA = nullptr, *MC = nullptr, *Yf = nullptr, *Zf = nullptr;
  size_t full_extra = 0;  // bytes of the tensor path's full-K scratch, admitted on first use
  // xk_coulomb (FP64 handles): allocated and admitted on first use
  double *Jrho = nullptr, *Jv = nullptr, *Jphiv = nullptr, *Jd = nullptr, *Jout = nullptr;
  double2 *Jc0 = nullptr, *Jc1 = nullptr, *Jtw = nullptr;
  int Jg = 0;
  double *C = nullptr, *psi = nullptr, *psig = nullptr, *V2 = nullptr, *M1 = nullptr,
         *M2 = nullptr, *Q = nullptr, *M3 = nullptr, *L1 = nullptr, *L2 = nullptr,
         *L3 = nullptr, *K = nullptr, *Ex = nullptr, *work = nullptr, *red = nullptr;
  // occ-RI K_ij factorisation scratch
  double *Kij = nullptr, *Lf = nullptr, *U = nullptr, *Y = nullptr, *xi = nullptr,
         *sgn = nullptr;
  int* status = nullptr;
  double ridge = 0.0;  // xk_setup_isdf: ridge added to X_gg (0 when none was needed)

  xk::MixedState* mixed = nullptr;
  Slot slots[kSlots];

  // one tensor-path build captured as a CUDA graph on first use (C in h->C,
  // K and E_x in h->K, h->Ex), replayed while step timing is off; dropped
  // when a launch argument changes (xk_set_wait_limit)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint64_t glaunches = 0;  // kernels in one replay
  bool graph_off = false;  // capture failed once: enqueue directly
  // step timing (xk_timing_enable / xk_timing_read)
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  double step_ms[XK_NSTEPS] = {0};
  uint64_t step_builds[XK_NSTEPS] = {0};
};

namespace {

std::mutex g_tickets_mu;
std::unordered_map<xk_ticket, std::pair<xk_handle*, int>> g_tickets;
xk_ticket g_next_ticket = 1;

struct Plan {
  size_t f64 = 0;   // doubles
  size_t i32 = 0;   // int32
  size_t work = 0;  // doubles of split-K work
};

// Doubles of split-K work the FP64 contractions need (a contraction that
// runs unsplit needs none); with ace_only, only the occ-RI K_ij products.
size_t max_work(int64_t Ng, int N, int n, int Naux, bool ace_only = false, int ga = -1) {
  const int ng = (int)Ng;
  if (ga < 0) ga = Naux;  // rows of V and W held (a shard's slice)
  size_t w = 1;
  auto acc = [&](int M, int Nc, int K) {
    const size_t ks = (size_t)xk::dgemm_ksplit(M, Nc, K);
    if (ks > 1) w = std::max(w, ks * (size_t)M * (size_t)Nc);
  };
  acc(n, n, N);         // K_ij
  acc(N, n, n);         // K U
  if (ace_only) return w;
  acc(ng, n, N);        // Psi = Phi C
  acc(ga, ng, n);       // V2 = V o (Psi_g Psi^T)
  acc(ga, n, ng);       // M2 = V2 Psi
  acc(n, ng, ga);       // M1 = Psi_g^T V2
  acc(n, N, ng);        // line1
  acc(n, N, ga);        // line2, line3
  acc(ga, Naux, n);     // W o Q
  acc(ga, n, Naux);     // M3
  acc(ga, N, ng);       // full K: M_A = V2 Phi
  acc(ga, N, Naux);     // full K: M_C = (W o Q) Phi_g
  acc(N, N, ga);        // full K: Phi_g^T M
  acc(N, N, ng);        // Coulomb J = Phi^T (v o Phi)
  acc(Naux, Naux, N);   // ISDF set-up: Phi_g Phi_g^T
  acc(Naux, ng, N);     // ISDF set-up: Phi_g Phi^T
  acc(Naux, Naux, ng);  // ISDF set-up: W = V chi^T
  return std::max(w, (size_t)Naux);  // the set-up also keeps the diagonal of X_gg here
}

// Rows ga of V and W held (ga = Naux unless a shard); Psi_g at all Naux points.
Plan plan_fp64(int64_t Ng, int N, int n, int Naux, int ga = -1) {
  Plan p;
  if (ga < 0) ga = Naux;
  const size_t ng = (size_t)Ng, na = (size_t)Naux, gs = (size_t)ga;
  p.f64 = ng * N + gs * N + gs * ng + gs * na       // Phi, Phi_g (slice), V, W rows
          + (size_t)N * n + ng * n + na * n         // C, Psi, Psi_g
          + gs * ng + (size_t)n * ng + gs * n       // V2, M1, M2
          + gs * na + gs * n + 3 * (size_t)n * N    // Q, M3, lines
          + (size_t)N * n + 2 + xk::reduce_work_elems()  // K, E_x and E_K, reduction
          + (size_t)N * n + 1                            // C and E_x of xk_energy
          + 2 * gs * N + 3 * (size_t)N * N                // full K: M_A, M_C, Y, Z, K
          + 3 * (size_t)n * n + 2 * (size_t)N * n + n;   // K_ij, L, U, Y, xi, sign
  p.work = max_work(Ng, N, n, Naux, false, ga);
  p.f64 += p.work;
  p.i32 = na + 2;
  return p;
}

size_t plan_bytes(const Plan& p) { return p.f64 * 8 + p.i32 * 4 + 64 * 256; }

bool valid_sizes(int64_t Ng, int32_t N, int32_t n, int32_t Naux) {
  return Ng > 0 && N > 0 && n > 0 && Naux > 0 && n <= N && (int64_t)Naux <= Ng &&
         Ng < (int64_t)1 << 31;
}

template <class T>
cudaError_t dalloc(xk_handle* h, T** p, size_t elems) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(elems, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

void fold_marks(xk_handle* h);

// The handle's captured build graph, if any (its stream is idle or the
// caller holds the handle's lock).
void drop_graph(xk_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->glaunches = 0;
}

void free_handle(xk_handle* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (Slot& s : h->slots) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.C) cudaFreeHost(s.C);
    if (s.K) cudaFreeHost(s.K);
    if (s.Ex) cudaFreeHost(s.Ex);
    if (s.st) cudaFreeHost(s.st);
  }
  drop_graph(h);
  if (h->mixed) xk::mixed_destroy(h->mixed);
  fold_marks(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->stream) cudaStreamDestroy(h->stream);
  unadmit_bytes(h->footprint);
  delete h;
}

// Status word of the tensor-path kernels of the builds enqueued so far on
// `s`: read and cleared in stream order (so a later build on the stream
// starts from zero), then waited for.  0 when none gave up.
int take_status(xk_handle* h, cudaStream_t s, cudaError_t* err) {
  *err = cudaSuccess;
  if (!h->mixed) return 0;
  int st[4] = {0, 0, 0, 0};
  int* dev = xk::mixed_status_ptr(h->mixed);
  cudaError_t e = cudaMemcpyAsync(st, dev, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, 16, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *err = e;
  return st[0];
}

// Records the start or the end of `step` when timing is on.
struct StepMark {
  xk_handle* h;
  int step;
  cudaEvent_t a = nullptr, b = nullptr;
  StepMark(xk_handle* hh, int st) : h(hh), step(st) {
    if (!h->timing) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h->stream);
  }
  ~StepMark() {
    if (!a) return;
    cudaEventRecord(b, h->stream);
    h->marks.push_back({step, {a, b}});
  }
};

// Begin (begin != 0) or end a step of the mixed path: same events as StepMark.
void step_hook(void* ctx, int step, int begin) {
  xk_handle* h = static_cast<xk_handle*>(ctx);
  static thread_local cudaEvent_t open[XK_NSTEPS] = {nullptr};
  if (begin) {
    cudaEventCreate(&open[step]);
    cudaEventRecord(open[step], h->stream);
  } else if (open[step]) {
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, h->stream);
    h->marks.push_back({step, {open[step], b}});
    open[step] = nullptr;
  }
}

void fold_marks(xk_handle* h) {
  for (auto& m : h->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.second.first, m.second.second) == cudaSuccess) {
      h->step_ms[m.first] += ms;
      h->step_builds[m.first] += 1;
    }
    cudaEventDestroy(m.second.first);
    cudaEventDestroy(m.second.second);
  }
  h->marks.clear();
}

// Enqueue one FP64 build on h->stream.  C is in h->C; results land in h->K, h->Ex.
int enqueue_fp64(xk_handle* h) {
  using xk::DGemm;
  cudaStream_t s = h->stream;
  const int ng = (int)h->Ng, N = h->N, n = h->n, na = h->Naux, ga = h->ga;
  const double* psl = h->psig + (size_t)h->g0 * n;  // Psi_g of the held slice
  auto G = [&](int M, int Nc, int K, const double* A, long lda, bool ta, const double* B, long ldb,
               bool tb, double* C, long ldc, const double* H, long ldh) {
    DGemm g{M, Nc, K, A, lda, ta, B, ldb, tb, C, ldc, 1.0, H, ldh, 0, h->work};
    return xk::dgemm(g, s);
  };
  {  // Eq. rpsEx step 1: orbitals on the grid and at the interpolation points.
    StepMark m(h, XK_STEP_ORBITALS);
    XK_CUDA(G(ng, n, N, h->phi, N, false, h->C, n, false, h->psi, n, nullptr, 0));
    XK_CUDA(xk::gather_rows_f64(h->psi, n, h->idx, na, n, h->psig, n, s));
  }
  {  // Steps 2-3: pair kernel at (R_g, R) and the Hadamard with V, fused.
    StepMark m(h, XK_STEP_PAIR);
    XK_CUDA(G(ga, ng, n, psl, n, false, h->psi, n, true, h->V2, ng, h->V, ng));
  }
  {  // Line 2, first contraction (order (a)): M2 = V2 Psi.
    StepMark m(h, XK_STEP_M2);
    XK_CUDA(G(ga, n, ng, h->V2, ng, false, h->psi, n, false, h->M2, n, nullptr, 0));
  }
  {  // Line 1, first contraction: M1 = Psi_g^T V2.
    StepMark m(h, XK_STEP_M1);
    XK_CUDA(G(n, ng, ga, psl, n, true, h->V2, ng, false, h->M1, ng, nullptr, 0));
  }
  {  // Line 1, contraction with the basis on the grid.
    StepMark m(h, XK_STEP_LINE1);
    XK_CUDA(G(n, N, ng, h->M1, ng, false, h->phi, N, false, h->L1, N, nullptr, 0));
  }
  {  // Line 2, contraction with the basis at R_g.
    StepMark m(h, XK_STEP_LINE2);
    XK_CUDA(G(n, N, ga, h->M2, n, true, h->phig, N, false, h->L2, N, nullptr, 0));
  }
  {  // Line 3: W o (Psi_g Psi_g^T) over the slice's rows and every g', then two contractions.
    StepMark m(h, XK_STEP_LINE3);
    XK_CUDA(G(ga, na, n, psl, n, false, h->psig, n, true, h->Q, na, h->W, na));
    XK_CUDA(G(ga, n, na, h->Q, na, false, h->psig, n, false, h->M3, n, nullptr, 0));
    XK_CUDA(G(n, N, ga, h->M3, n, true, h->phig, N, false, h->L3, N, nullptr, 0));
  }
  {  // K_{mu i} = dV (line1 + line2 - line3)^T and E_x = -sum K o C.
    StepMark m(h, XK_STEP_ASSEMBLE);
    XK_CUDA(xk::assemble_k_f64(h->L1, h->L2, h->L3, n, N, h->dV, h->K, s));
    XK_CUDA(xk::neg_dot_f64(h->K, h->C, (long)N * n, h->red, h->Ex, s));
  }
  return XK_OK;
}

// Enqueue E_x alone from h->Ce into h->Ce[N n] (the closed form of E_x:
// -dV (2 sum V o P o P - sum W o Q o Q), no K).
int enqueue_energy(xk_handle* h) {
  double* Ex = h->Ce + (size_t)h->N * h->n;
  if (h->mode != XK_FP64) {
    xk::StepHook hook{h->timing ? &step_hook : nullptr, h};
    cudaError_t e = xk::mixed_enqueue_energy(h->mixed, h->Ce, Ex, h->stream, hook);
    if (e != cudaSuccess) return cuda_fail(e, "mixed-precision energy");
    return XK_OK;
  }
  using xk::DGemm;
  cudaStream_t s = h->stream;
  const int ng = (int)h->Ng, N = h->N, n = h->n, na = h->Naux, ga = h->ga;
  const double* psl = h->psig + (size_t)h->g0 * n;  // Psi_g of the held slice
  auto G = [&](int M, int Nc, int K, const double* A, long lda, bool ta, const double* B, long ldb,
               bool tb, double* C, long ldc) {
    DGemm g{M, Nc, K, A, lda, ta, B, ldb, tb, C, ldc, 1.0, nullptr, 0, 0, h->work};
    return xk::dgemm(g, s);
  };
  {
    StepMark m(h, XK_STEP_ORBITALS);
    XK_CUDA(G(ng, n, N, h->phi, N, false, h->Ce, n, false, h->psi, n));
    XK_CUDA(xk::gather_rows_f64(h->psi, n, h->idx, na, n, h->psig, n, s));
  }
  {  // P = Psi_g Psi^T and Q = Psi_g Psi_g^T
    StepMark m(h, XK_STEP_PAIR);
    XK_CUDA(G(ga, ng, n, psl, n, false, h->psi, n, true, h->V2, ng));
    XK_CUDA(G(ga, na, n, psl, n, false, h->psig, n, true, h->Q, na));
  }
  {
    StepMark m(h, XK_STEP_ASSEMBLE);
    XK_CUDA(xk::closed_form_ex_f64(h->V, h->V2, (long)ga * ng, h->W, h->Q, (long)ga * na, h->dV,
                                   h->red, Ex, s));
  }
  return XK_OK;
}

// Enqueue K_{mu nu} (Eq. rpsEx, all three terms of Eq. rps) from h->Ce into h->Kf.
int enqueue_full(xk_handle* h) {
  if (h->mode != XK_FP64) {
    xk::StepHook hook{h->timing ? &step_hook : nullptr, h};
    cudaError_t e = xk::mixed_enqueue_full(h->mixed, h->Ce, h->Kf, h->stream, hook);
    if (e != cudaSuccess) return cuda_fail(e, "mixed-precision full K");
    return XK_OK;
  }
  using xk::DGemm;
  cudaStream_t s = h->stream;
  const int ng = (int)h->Ng, N = h->N, n = h->n, na = h->Naux;
  auto G = [&](int M, int Nc, int K, const double* A, long lda, bool ta, const double* B, long ldb,
               bool tb, double* C, long ldc, const double* H, long ldh) {
    DGemm g{M, Nc, K, A, lda, ta, B, ldb, tb, C, ldc, 1.0, H, ldh, 0, h->work};
    return xk::dgemm(g, s);
  };
  {
    StepMark m(h, XK_STEP_ORBITALS);
    XK_CUDA(G(ng, n, N, h->phi, N, false, h->Ce, n, false, h->psi, n, nullptr, 0));
    XK_CUDA(xk::gather_rows_f64(h->psi, n, h->idx, na, n, h->psig, n, s));
  }
  {  // V2 = V o (Psi_g Psi^T), M_A = V2 Phi
    StepMark m(h, XK_STEP_PAIR);
    XK_CUDA(G(na, ng, n, h->psig, n, false, h->psi, n, true, h->V2, ng, h->V, ng));
    XK_CUDA(G(na, N, ng, h->V2, ng, false, h->phi, N, false, h->MA, N, nullptr, 0));
  }
  {  // W o (Psi_g Psi_g^T), M_C = (W o Q) Phi_g
    StepMark m(h, XK_STEP_LINE3);
    XK_CUDA(G(na, na, n, h->psig, n, false, h->psig, n, true, h->Q, na, h->W, na));
    XK_CUDA(G(na, N, na, h->Q, na, false, h->phig, N, false, h->MC, N, nullptr, 0));
  }
  {  // Y = Phi_g^T M_A, Z = Phi_g^T M_C, K = dV (Y + Y^T - Z)
    StepMark m(h, XK_STEP_ASSEMBLE);
    XK_CUDA(G(N, N, na, h->phig, N, true, h->MA, N, false, h->Yf, N, nullptr, 0));
    XK_CUDA(G(N, N, na, h->phig, N, true, h->MC, N, false, h->Zf, N, nullptr, 0));
    XK_CUDA(xk::assemble_full_f64(h->Yf, h->Zf, N, h->dV, h->Kf, s));
  }
  return XK_OK;
}

// Ex[0] = E_x; Ex[1] = -sum K o C of the K the build returns.  On the FP64
// path the two are the same number; on the tensor path E_x is the closed
// form (pin P8) and the gap |Ex[0] - Ex[1]| is the build's error estimate.
int enqueue_build(xk_handle* h) {
  if (h->mode == XK_FP64) {
    int rc = enqueue_fp64(h);
    if (rc != XK_OK) return rc;
    XK_CUDA(cudaMemcpyAsync(h->Ex + 1, h->Ex, 8, cudaMemcpyDeviceToDevice, h->stream));
    return XK_OK;
  }
  if (!h->timing && !h->graph_off && !std::getenv("XK_NO_GRAPH") &&
      (h->gexec || g_setups_running.load() == 0)) {
    // the whole device part of a build as one graph: one launch from the
    // host instead of ~25, and no gaps between the kernels
    if (!h->gexec) {
      const uint64_t l0 = xk::t_launches;
      xk::StepHook none{nullptr, nullptr};
      cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        e = xk::mixed_enqueue(h->mixed, h->C, h->K, h->Ex, h->stream, none);
        if (e == cudaSuccess)
          e = xk::neg_dot_f64(h->K, h->C, (long)h->N * h->n, h->red, h->Ex + 1, h->stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
        if (e == cudaSuccess) e = ec;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, graph, 0);
        if (e == cudaSuccess) {
          h->graph = graph;
        } else if (graph) {
          cudaGraphDestroy(graph);
        }
      }
      const uint64_t captured = xk::t_launches - l0;
      xk::g_launches.fetch_sub(captured);  // counted per replay below
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        h->gexec = nullptr;
        h->graph_off = true;  // enqueue directly from now on
      } else {
        h->glaunches = captured;
      }
    }
    if (h->gexec) {
      XK_CUDA(cudaGraphLaunch(h->gexec, h->stream));
      xk::g_launches.fetch_add(h->glaunches);
      return XK_OK;
    }
  }
  xk::StepHook hook{h->timing ? &step_hook : nullptr, h};
  cudaError_t e = xk::mixed_enqueue(h->mixed, h->C, h->K, h->Ex, h->stream, hook);
  if (e == cudaSuccess)
    e = xk::neg_dot_f64(h->K, h->C, (long)h->N * h->n, h->red, h->Ex + 1, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mixed-precision build");
  return XK_OK;
}

}  // namespace

extern "C" {

const char* xk_last_error(void) { return t_err.c_str(); }

uint64_t xk_kernel_launches(void) { return xk::g_launches.load(); }

int xk_footprint(int64_t Ng, int32_t N, int32_t n, int32_t Naux, int mode, size_t* bytes) {
  if (!bytes) return fail(XK_EINVAL, "xk_footprint: bytes is NULL");
  if (!valid_sizes(Ng, N, n, Naux)) return fail(XK_EINVAL, "xk_footprint: invalid sizes");
  if (mode == XK_FP64) {
    *bytes = plan_bytes(plan_fp64(Ng, N, n, Naux));
    return XK_OK;
  }
  if (mode == XK_F16X3) {
    *bytes = xk::mixed_footprint(Ng, N, n, Naux, Naux) + (size_t)N * n * 8 * 3 + 16 + (size_t)N * N * 8 +
             (size_t)max_work(Ng, N, n, Naux, true) * 8 + 4 * (size_t)n * n * 8 + 2 * (size_t)N * n * 8 +
             65536;
    return XK_OK;
  }
  return fail(XK_EINVAL, "xk_footprint: unknown mode");
}

// xk_setup (V, W given) and xk_setup_isdf (V == W == nullptr: chi, V and W
// formed on the device from phi and idx on a cubic grid^3 grid of side L).
// A shard (xk_setup_shard) holds the rows [g0, g1) of V and W; V and W then
// point at those g1 - g0 rows (V: N_g columns, W: all Naux columns).
static int setup_impl(int64_t Ng, int32_t N, int32_t n, int32_t Naux, const double* phi,
               const int32_t* idx, const double* V, const double* W, double dV, int mode,
               int32_t grid, double L, xk_handle** out, int32_t g0 = 0, int32_t g1 = -1,
               double queue_ms = -1.0) {
  if (!out) return fail(XK_EINVAL, "xk_setup: out is NULL");
  *out = nullptr;
  const SetupMark running;  // builds elsewhere defer their graph capture meanwhile
  if (g1 < 0) g1 = Naux;
  const bool isdf = V == nullptr && W == nullptr && grid > 0;
  if (!phi || !idx || (!isdf && (!V || !W))) return fail(XK_EINVAL, "xk_setup: NULL table pointer");
  if (!valid_sizes(Ng, N, n, Naux)) return fail(XK_EINVAL, "xk_setup: invalid sizes");
  if (g0 < 0 || g1 > Naux || g0 >= g1)
    return fail(XK_EINVAL, "xk_setup_shard: the slice [g0, g1) must be non-empty within [0, Naux)");
  const int32_t ga = g1 - g0;
  if (!(dV > 0.0) || !std::isfinite(dV)) return fail(XK_EINVAL, "xk_setup: dV must be > 0");
  if (mode != XK_FP64 && mode != XK_F16X3) return fail(XK_EINVAL, "xk_setup: unsupported mode");
  {
    std::vector<int32_t> s(idx, idx + Naux);
    std::sort(s.begin(), s.end());
    if (s.front() < 0 || (int64_t)s.back() >= Ng)
      return fail(XK_EINVAL, "xk_setup: interp_idx out of range");
    if (std::adjacent_find(s.begin(), s.end()) != s.end())
      return fail(XK_EINVAL, "xk_setup: interp_idx has duplicates");
  }
  if (!isdf) {
    // W is symmetric: checked on the block of the held rows [g0, g1) x [g0, g1)
    double wmax = 0.0, asym = 0.0;
    const size_t na = (size_t)Naux, gs = (size_t)ga;
    for (size_t i = 0; i < gs; ++i)
      for (size_t j = 0; j < na; ++j) {
        const double a = W[i * na + j];
        if (!std::isfinite(a)) return fail(XK_EINVAL, "xk_setup: W has non-finite entries");
        wmax = std::max(wmax, std::fabs(a));
        if (j >= (size_t)g0 && j - g0 > i && j - g0 < gs)
          asym = std::max(asym, std::fabs(a - W[(j - g0) * na + g0 + i]));
      }
    if (asym > 1e-12 * wmax) return fail(XK_EINVAL, "xk_setup: W_aux is not symmetric");
  }
  size_t need = 0;
  int rc = xk_footprint(Ng, N, n, Naux, mode, &need);
  if (rc != XK_OK) return rc;
  if (ga != Naux)  // a shard holds the slice's rows only
    need = mode == XK_FP64 ? plan_bytes(plan_fp64(Ng, N, n, Naux, ga))
                           : xk::mixed_footprint(Ng, N, n, ga, Naux) + (size_t)N * n * 8 * 3 + 16 +
                                 (size_t)N * N * 8 + (size_t)max_work(Ng, N, n, Naux, true) * 8 +
                                 4 * (size_t)n * n * 8 + 2 * (size_t)N * n * 8 + 65536;
  // the tensor path's ISDF set-up holds FP64 temporaries next to its tables:
  // Phi, Phi_g, X_gg, chi, V, W and the product work (freed before return)
  const size_t isdf_tmp = (isdf && mode != XK_FP64)
      ? ((size_t)Ng * N + (size_t)Naux * N + 2 * (size_t)Naux * Naux + 2 * (size_t)Naux * Ng +
         max_work(Ng, N, n, Naux) + (size_t)Naux) * 8 + (size_t)Naux * 4
      : 0;

  // admission: now (queue_ms < 0) or in arrival order within queue_ms
  {
    int rc = admit_bytes(need + isdf_tmp, queue_ms, true, "xk_setup");
    if (rc != XK_OK) return rc;
  }
  int dev = 0;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      unadmit_bytes(need + isdf_tmp);
      return cuda_fail(e, "cudaGetDevice");
    }
  }

  xk_handle* h = new xk_handle();
  h->Ng = Ng; h->N = N; h->n = n; h->Naux = Naux; h->dV = dV; h->mode = mode; h->device = dev;
  h->g0 = g0; h->ga = ga;
  h->footprint = need + isdf_tmp;  // the ISDF temporaries are returned at the end
  auto bail = [&](int code) { free_handle(h); return code; };
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));

  const size_t ng = (size_t)Ng, na = (size_t)Naux;
#define XK_ALLOC(ptr, elems)                                  \
  do {                                                        \
    cudaError_t e_ = dalloc(h, &(ptr), (elems));              \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, "cudaMalloc " #ptr)); \
  } while (0)
  XK_ALLOC(h->C, (size_t)N * n);
  XK_ALLOC(h->Ce, (size_t)N * n + 1);
  XK_ALLOC(h->Kf, (size_t)N * N);
  XK_ALLOC(h->K, (size_t)N * n);
  XK_ALLOC(h->Ex, 2);  // E_x and the energy of the returned K, -sum K o C
  XK_ALLOC(h->Kij, (size_t)n * n);
  XK_ALLOC(h->Lf, (size_t)n * n);
  XK_ALLOC(h->U, (size_t)n * n);
  XK_ALLOC(h->Y, (size_t)N * n);
  XK_ALLOC(h->xi, (size_t)N * n);
  XK_ALLOC(h->sgn, (size_t)n);
  XK_ALLOC(h->status, 2);
  XK_ALLOC(h->red, xk::reduce_work_elems());
  const size_t work = max_work(Ng, N, n, Naux, mode != XK_FP64, ga);
  XK_ALLOC(h->work, work);
  if (mode == XK_FP64) {
    const size_t gs = (size_t)ga;  // rows of V, W, P and Q held
    XK_ALLOC(h->phi, ng * N);
    XK_ALLOC(h->phig, gs * N);
    XK_ALLOC(h->V, gs * ng);
    XK_ALLOC(h->W, gs * na);
    XK_ALLOC(h->idx, na);
    XK_ALLOC(h->psi, ng * n);
    XK_ALLOC(h->psig, na * n);
    XK_ALLOC(h->V2, gs * ng);
    XK_ALLOC(h->M1, (size_t)n * ng);
    XK_ALLOC(h->M2, gs * n);
    XK_ALLOC(h->Q, gs * na);
    XK_ALLOC(h->M3, gs * n);
    XK_ALLOC(h->L1, (size_t)n * N);
    XK_ALLOC(h->L2, (size_t)n * N);
    XK_ALLOC(h->L3, (size_t)n * N);
    XK_ALLOC(h->MA, gs * N);
    XK_ALLOC(h->MC, gs * N);
    XK_ALLOC(h->Yf, (size_t)N * N);
    XK_ALLOC(h->Zf, (size_t)N * N);
    e = cudaMemcpyAsync(h->phi, phi, ng * N * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !isdf)
      e = cudaMemcpyAsync(h->V, V, gs * ng * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !isdf)
      e = cudaMemcpyAsync(h->W, W, gs * na * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->idx, idx, na * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)  // the basis at the slice's points
      e = xk::gather_rows_f64(h->phi, N, h->idx + g0, ga, N, h->phig, N, h->stream);
    if (e == cudaSuccess && isdf)  // X_gg in Q, chi in V2 (both scratch of the build)
      e = xk::isdf_tables_f64(h->phi, (long)ng, N, h->phig, Naux, grid, L, h->Q, h->V2, h->V, h->W,
                              h->work, h->status, &h->ridge, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaErrorInvalidValue && isdf)
      return bail(fail(XK_EINVAL, "xk_setup_isdf: X_gg is not positive definite even with the ridge"));
    if (e != cudaSuccess) return bail(cuda_fail(e, "xk_setup upload"));
  } else {
    if (isdf) {  // FP64 tables on the device first, then the tensor path's own tables
      std::vector<void*> tmp;
      auto talloc = [&](double** p, size_t elems) {
        void* q = nullptr;
        cudaError_t r = cudaMalloc(&q, std::max<size_t>(elems, 1) * 8);
        if (r == cudaSuccess) tmp.push_back(q);
        *p = static_cast<double*>(q);
        return r;
      };
      auto release = [&]() {
        for (void* q : tmp) cudaFree(q);
        tmp.clear();
      };
      double *dphi = nullptr, *dphig = nullptr, *Xgg = nullptr, *chi = nullptr, *dV_ = nullptr,
             *dW = nullptr, *wk = nullptr, *didx = nullptr;
      e = talloc(&dphi, ng * N);
      if (e == cudaSuccess) e = talloc(&dphig, na * N);
      if (e == cudaSuccess) e = talloc(&Xgg, na * na);
      if (e == cudaSuccess) e = talloc(&chi, na * ng);
      if (e == cudaSuccess) e = talloc(&dV_, na * ng);
      if (e == cudaSuccess) e = talloc(&dW, na * na);
      if (e == cudaSuccess) e = talloc(&wk, std::max(max_work(Ng, N, n, Naux), na));
      if (e == cudaSuccess) e = talloc(&didx, (na + 1) / 2);
      int32_t* di = reinterpret_cast<int32_t*>(didx);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dphi, phi, ng * N * 8, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(di, idx, na * 4, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = xk::gather_rows_f64(dphi, N, di, Naux, N, dphig, N, h->stream);
      if (e == cudaSuccess)
        e = xk::isdf_tables_f64(dphi, (long)ng, N, dphig, Naux, grid, L, Xgg, chi, dV_, dW, wk,
                                h->status, &h->ridge, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e == cudaSuccess) {  // chi and X_gg are no longer needed
        cudaFree(chi); cudaFree(Xgg);
        tmp.erase(std::remove_if(tmp.begin(), tmp.end(),
                                 [&](void* q) { return q == chi || q == Xgg; }), tmp.end());
        e = xk::mixed_create(Ng, N, n, Naux, 0, Naux, dphi, idx, dV_, dW, dV, h->stream, &h->mixed);
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, 8, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      release();
    } else {
      e = xk::mixed_create(Ng, N, n, Naux, g0, g1, phi, idx, V, W, dV, h->stream, &h->mixed);
    }
    if (e == cudaErrorInvalidValue)
      return bail(fail(XK_EINVAL, "xk_setup: basis columns are linearly dependent on the grid"));
    if (e != cudaSuccess) return bail(cuda_fail(e, "xk_setup mixed tables"));
  }
#undef XK_ALLOC
  for (Slot& s : h->slots) {
    e = cudaHostAlloc((void**)&s.C, (size_t)N * n * 8, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s.K, (size_t)N * n * 8, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s.Ex, 16, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s.st, 16, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "xk_setup slots"));
  }
  if (isdf_tmp) {  // the ISDF set-up's temporaries are freed: return their bytes
    h->footprint = need;
    unadmit_bytes(isdf_tmp);
  }
  *out = h;
  return XK_OK;
}

int xk_setup(int64_t Ng, int32_t N, int32_t n, int32_t Naux, const double* phi,
             const int32_t* idx, const double* V, const double* W, double dV, int mode,
             xk_handle** out) {
  if (!V || !W) {
    if (out) *out = nullptr;
    return fail(XK_EINVAL, "xk_setup: NULL table pointer");
  }
  return setup_impl(Ng, N, n, Naux, phi, idx, V, W, dV, mode, 0, 0.0, out);
}

int xk_setup_shard(int64_t Ng, int32_t N, int32_t n, int32_t Naux, int32_t g0, int32_t g1,
                   const double* basis_on_points, const int32_t* interp_idx,
                   const double* V_rows, const double* W_rows, double dV, int mode,
                   xk_handle** out) {
  if (!V_rows || !W_rows) {
    if (out) *out = nullptr;
    return fail(XK_EINVAL, "xk_setup_shard: NULL table pointer");
  }
  return setup_impl(Ng, N, n, Naux, basis_on_points, interp_idx, V_rows, W_rows, dV, mode, 0, 0.0,
                    out, g0, g1);
}

int xk_setup_queued(int64_t Ng, int32_t N, int32_t n, int32_t Naux, const double* phi,
                    const int32_t* idx, const double* V, const double* W, double dV, int mode,
                    double timeout_ms, xk_handle** out) {
  if (!V || !W) {
    if (out) *out = nullptr;
    return fail(XK_EINVAL, "xk_setup_queued: NULL table pointer");
  }
  if (!(timeout_ms >= 0.0) || !std::isfinite(timeout_ms)) {
    if (out) *out = nullptr;
    return fail(XK_EINVAL, "xk_setup_queued: timeout_ms must be finite and >= 0");
  }
  return setup_impl(Ng, N, n, Naux, phi, idx, V, W, dV, mode, 0, 0.0, out, 0, -1, timeout_ms);
}

int xk_admit_reserve(uint64_t bytes, double timeout_ms, uint64_t* token) {
  if (!token) return fail(XK_EINVAL, "xk_admit_reserve: token is NULL");
  *token = 0;
  if (!std::isfinite(timeout_ms)) return fail(XK_EINVAL, "xk_admit_reserve: timeout_ms is not finite");
  // without XK_HBM_BUDGET_BYTES the budget is the current device's free memory
  const bool device = std::getenv("XK_HBM_BUDGET_BYTES") == nullptr;
  int rc = admit_bytes((size_t)bytes, timeout_ms, device, "xk_admit_reserve");
  if (rc != XK_OK) return rc;
  std::lock_guard<std::mutex> lk(g_admit_mu);
  const uint64_t t = ++g_admit_seq;
  g_reservations[t] = (size_t)bytes;
  g_reserved += (size_t)bytes;
  *token = t;
  return XK_OK;
}

int xk_admit_release(uint64_t token) {
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(g_admit_mu);
    auto it = g_reservations.find(token);
    if (it == g_reservations.end()) return fail(XK_EINVAL, "xk_admit_release: unknown token");
    bytes = it->second;
    g_reserved -= std::min(g_reserved, bytes);
    g_reservations.erase(it);
  }
  unadmit_bytes(bytes);
  return XK_OK;
}

int xk_admit_state(uint64_t* admitted_bytes, uint32_t* waiting) {
  if (!admitted_bytes || !waiting) return fail(XK_EINVAL, "xk_admit_state: NULL argument");
  std::lock_guard<std::mutex> lk(g_admit_mu);
  *admitted_bytes = (uint64_t)g_admitted;
  *waiting = (uint32_t)g_admit_queue.size();
  return XK_OK;
}

int xk_setup_isdf(int64_t Ng, int32_t N, int32_t n, int32_t Naux, const double* phi,
                  const int32_t* idx, int32_t grid, double L, int mode, xk_handle** out) {
  if (out) *out = nullptr;
  if (grid <= 0 || (int64_t)grid * grid * grid != Ng)
    return fail(XK_EINVAL, "xk_setup_isdf: grid^3 must equal N_g");
  if (!(L > 0.0) || !std::isfinite(L)) return fail(XK_EINVAL, "xk_setup_isdf: L must be > 0");
  return setup_impl(Ng, N, n, Naux, phi, idx, nullptr, nullptr, L * L * L / (double)Ng, mode, grid,
                    L, out);
}

int xk_isdf_points(int32_t m, int32_t N, const double* rows, int32_t want, double tol_rel,
                   int32_t* piv_out, int32_t* count) {
  if (!rows || !piv_out || !count) return fail(XK_EINVAL, "xk_isdf_points: NULL argument");
  if (m <= 0 || N <= 0 || want <= 0) return fail(XK_EINVAL, "xk_isdf_points: invalid sizes");
  if (!(tol_rel >= 0.0) || !std::isfinite(tol_rel))
    return fail(XK_EINVAL, "xk_isdf_points: tol_rel must be finite and >= 0");
  const size_t need = ((size_t)m * m + (size_t)m * std::min(want, m) + (size_t)m * N + 2 * (size_t)m) * 8;
  size_t freeb = 0, totalb = 0;
  XK_CUDA(cudaMemGetInfo(&freeb, &totalb));
  {
    std::lock_guard<std::mutex> al(g_admit_mu);
    const size_t reserve = (size_t)1 << 30;
    size_t budget = freeb > reserve ? freeb - reserve : 0;
    if (const char* env = std::getenv("XK_HBM_BUDGET_BYTES")) {
      const size_t cap = (size_t)std::strtoull(env, nullptr, 10);
      budget = std::min(budget, cap > g_admitted ? cap - g_admitted : 0);
    }
    if (need > budget)
      return fail(XK_ENOMEM, "xk_isdf_points: scratch of " + std::to_string(need) +
                                 " bytes exceeds the admission budget " + std::to_string(budget));
  }
  cudaStream_t s = nullptr;
  XK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double* F = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&F), (size_t)m * N * 8, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F, rows, (size_t)m * N * 8, cudaMemcpyHostToDevice, s);
  int got = 0;
  if (e == cudaSuccess) e = xk::select_points_f64(F, m, N, want, tol_rel, piv_out, &got, s);
  if (F) cudaFreeAsync(F, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "xk_isdf_points");
  *count = got;
  return XK_OK;
}

int xk_tables(xk_handle* h, double* W_out, const int32_t* rows, int32_t nrows, double* V_rows_out,
              double* ridge) {
  if (!h) return fail(XK_EINVAL, "xk_tables: NULL handle");
  if (h->mode != XK_FP64) return fail(XK_EINVAL, "xk_tables: needs an XK_FP64 handle");
  if (h->ga != h->Naux) return fail(XK_EINVAL, "xk_tables: not for a shard handle");
  if (nrows < 0 || (nrows > 0 && (!rows || !V_rows_out)))
    return fail(XK_EINVAL, "xk_tables: bad row list");
  for (int32_t i = 0; i < nrows; ++i)
    if (rows[i] < 0 || rows[i] >= h->Naux) return fail(XK_EINVAL, "xk_tables: row out of range");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  const size_t na = (size_t)h->Naux, ng = (size_t)h->Ng;
  if (W_out) XK_CUDA(cudaMemcpyAsync(W_out, h->W, na * na * 8, cudaMemcpyDeviceToHost, h->stream));
  for (int32_t i = 0; i < nrows; ++i)
    XK_CUDA(cudaMemcpyAsync(V_rows_out + (size_t)i * ng, h->V + (size_t)rows[i] * ng, ng * 8,
                            cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaStreamSynchronize(h->stream));
  if (ridge) *ridge = h->ridge;
  return XK_OK;
}

int xk_build_device(xk_handle* h, const double* C_dev, double* K_dev, double* Ex_dev,
                    void* stream) {
  if (!h || !C_dev || !K_dev || !Ex_dev) return fail(XK_EINVAL, "xk_build_device: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  const size_t kb = (size_t)h->N * h->n * 8;
  // Order the handle's stream after the caller's stream, run, then order back.
  cudaEvent_t ev;
  XK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  XK_CUDA(cudaEventRecord(ev, us));
  XK_CUDA(cudaStreamWaitEvent(h->stream, ev, 0));
  XK_CUDA(cudaMemcpyAsync(h->C, C_dev, kb, cudaMemcpyDeviceToDevice, h->stream));
  int rc = enqueue_build(h);
  if (rc != XK_OK) { cudaEventDestroy(ev); return rc; }
  XK_CUDA(cudaMemcpyAsync(K_dev, h->K, kb, cudaMemcpyDeviceToDevice, h->stream));
  XK_CUDA(cudaMemcpyAsync(Ex_dev, h->Ex, 8, cudaMemcpyDeviceToDevice, h->stream));
  XK_CUDA(cudaEventRecord(ev, h->stream));
  XK_CUDA(cudaStreamWaitEvent(us, ev, 0));
  cudaEventDestroy(ev);
  h->has_build = true;
  return XK_OK;
}

int xk_build(xk_handle* h, const double* C, double* K_out, double* Ex) {
  if (!h || !C || !K_out || !Ex) return fail(XK_EINVAL, "xk_build: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  const size_t kb = (size_t)h->N * h->n * 8;
  XK_CUDA(cudaMemcpyAsync(h->C, C, kb, cudaMemcpyHostToDevice, h->stream));
  int rc = enqueue_build(h);
  if (rc != XK_OK) return rc;
  XK_CUDA(cudaMemcpyAsync(K_out, h->K, kb, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaMemcpyAsync(Ex, h->Ex, 8, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaStreamSynchronize(h->stream));
  h->has_build = true;
  {
    cudaError_t e = cudaSuccess;
    const int st = take_status(h, h->stream, &e);
    if (e != cudaSuccess) return cuda_fail(e, "xk_build status");
    if (st != 0)
      return fail(XK_ETIMEDOUT, "xk_build: a bounded wait inside a kernel gave up (code " +
                                    std::to_string(st) + ")");
  }
  return XK_OK;
}

int xk_build_full(xk_handle* h, const double* C, double* K_out) {
  if (!h || !C || !K_out) return fail(XK_EINVAL, "xk_build_full: NULL argument");
  if (h->ga != h->Naux) return fail(XK_EINVAL, "xk_build_full: not for a shard handle");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  if (h->mode != XK_FP64 && h->full_extra == 0) {
    // first use on the tensor path: admit and allocate the full-K scratch
    const size_t extra = xk::mixed_full_footprint(h->Ng, h->N, h->n, h->Naux);
    size_t freeb = 0, totalb = 0;
    XK_CUDA(cudaMemGetInfo(&freeb, &totalb));
    {
      std::lock_guard<std::mutex> al(g_admit_mu);
      const size_t reserve = (size_t)1 << 30;
      size_t budget = freeb > reserve ? freeb - reserve : 0;
      if (const char* env = std::getenv("XK_HBM_BUDGET_BYTES")) {
        const size_t cap = (size_t)std::strtoull(env, nullptr, 10);
        budget = std::min(budget, cap > g_admitted ? cap - g_admitted : 0);
      }
      if (extra > budget)
        return fail(XK_ENOMEM, "xk_build_full: full-K scratch of " + std::to_string(extra) +
                                   " bytes exceeds the admission budget " + std::to_string(budget));
      g_admitted += extra;
    }
    h->full_extra = extra;
    h->footprint += extra;
    cudaError_t e = xk::mixed_full_prepare(h->mixed);
    if (e != cudaSuccess) return cuda_fail(e, "xk_build_full scratch");
  }
  XK_CUDA(cudaMemcpyAsync(h->Ce, C, (size_t)h->N * h->n * 8, cudaMemcpyHostToDevice, h->stream));
  int rc = enqueue_full(h);
  if (rc != XK_OK) return rc;
  XK_CUDA(cudaMemcpyAsync(K_out, h->Kf, (size_t)h->N * h->N * 8, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaStreamSynchronize(h->stream));
  {
    cudaError_t e = cudaSuccess;
    const int st = take_status(h, h->stream, &e);
    if (e != cudaSuccess) return cuda_fail(e, "xk_build_full status");
    if (st != 0)
      return fail(XK_ETIMEDOUT, "xk_build_full: a bounded wait inside a kernel gave up (code " +
                                    std::to_string(st) + ")");
  }
  return XK_OK;
}

int xk_coulomb(xk_handle* h, int32_t grid, double L, const double* C, double* J_out,
               double* E_J) {
  if (!h || !C || !J_out || !E_J) return fail(XK_EINVAL, "xk_coulomb: NULL argument");
  if (h->mode != XK_FP64)
    return fail(XK_EINVAL, "xk_coulomb: needs an XK_FP64 handle (the FP64 basis table)");
  if (grid <= 0 || (int64_t)grid * grid * grid != h->Ng)
    return fail(XK_EINVAL, "xk_coulomb: grid^3 must equal N_g");
  if (!(L > 0.0) || !std::isfinite(L)) return fail(XK_EINVAL, "xk_coulomb: L must be > 0");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  cudaStream_t s = h->stream;
  const int N = h->N, n = h->n;
  const size_t ng = (size_t)h->Ng;
  if (h->Jg == 0) {  // first use: admit and allocate the scratch
    const size_t extra = (ng * (size_t)N + 2 * ng + 4 * ng + (size_t)N * N + 1 + 2 * (size_t)grid) * 8;
    size_t freeb = 0, totalb = 0;
    XK_CUDA(cudaMemGetInfo(&freeb, &totalb));
    {
      std::lock_guard<std::mutex> al(g_admit_mu);
      const size_t reserve = (size_t)1 << 30;
      size_t budget = freeb > reserve ? freeb - reserve : 0;
      if (const char* env = std::getenv("XK_HBM_BUDGET_BYTES")) {
        const size_t cap = (size_t)std::strtoull(env, nullptr, 10);
        budget = std::min(budget, cap > g_admitted ? cap - g_admitted : 0);
      }
      if (extra > budget)
        return fail(XK_ENOMEM, "xk_coulomb: scratch of " + std::to_string(extra) +
                                   " bytes exceeds the admission budget " + std::to_string(budget));
      g_admitted += extra;
    }
    h->footprint += extra;
    auto A = [&](double** p, size_t elems) { return dalloc(h, p, elems); };
    XK_CUDA(A(&h->Jphiv, ng * N));
    XK_CUDA(A(&h->Jrho, ng));
    XK_CUDA(A(&h->Jv, ng));
    double* cbuf = nullptr;
    XK_CUDA(A(&cbuf, 4 * ng));
    h->Jc0 = reinterpret_cast<double2*>(cbuf);
    h->Jc1 = h->Jc0 + ng;
    XK_CUDA(A(&h->Jout, (size_t)N * N + 1));
    double* tw = nullptr;
    XK_CUDA(A(&tw, 2 * (size_t)grid));
    h->Jtw = reinterpret_cast<double2*>(tw);
    std::vector<double> t(2 * (size_t)grid);
    for (int m = 0; m < grid; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)grid;
      t[2 * m] = std::cos(a);
      t[2 * m + 1] = std::sin(a);
    }
    XK_CUDA(cudaMemcpyAsync(tw, t.data(), t.size() * 8, cudaMemcpyHostToDevice, s));
    XK_CUDA(cudaStreamSynchronize(s));
    h->Jg = grid;
  }
  XK_CUDA(cudaMemcpyAsync(h->Ce, C, (size_t)N * n * 8, cudaMemcpyHostToDevice, s));
  {
    StepMark m(h, XK_STEP_ORBITALS);
    xk::DGemm g1{(int)ng, n, N, h->phi, N, false, h->Ce, n, false, h->psi, n, 1.0, nullptr, 0, 0, h->work};
    XK_CUDA(xk::dgemm(g1, s));
  }
  {  // density, Poisson solve, J = dV Phi^T (v o Phi), E_J = dV sum rho v
    StepMark m(h, XK_STEP_PAIR);
    XK_CUDA(xk::coulomb_potential_f64(h->psi, (long)ng, n, grid, L, h->Jtw, h->Jrho, h->Jc0, h->Jc1, s));
    XK_CUDA(xk::potential_rows_f64(h->Jc0, h->phi, (long)ng, N, h->Jv, h->Jphiv, s));
    xk::DGemm gj{N, N, (int)ng, h->phi, N, true, h->Jphiv, N, false, h->Jout, N, h->dV, nullptr, 0, 0, h->work};
    XK_CUDA(xk::dgemm(gj, s));
    XK_CUDA(xk::dot_f64(h->Jrho, h->Jv, (long)ng, h->dV, h->red, h->Jout + (size_t)N * N, s));
  }
  XK_CUDA(cudaMemcpyAsync(J_out, h->Jout, (size_t)N * N * 8, cudaMemcpyDeviceToHost, s));
  XK_CUDA(cudaMemcpyAsync(E_J, h->Jout + (size_t)N * N, 8, cudaMemcpyDeviceToHost, s));
  XK_CUDA(cudaStreamSynchronize(s));
  return XK_OK;
}

int xk_energy(xk_handle* h, const double* C, double* Ex) {
  if (!h || !C || !Ex) return fail(XK_EINVAL, "xk_energy: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  const size_t cb = (size_t)h->N * h->n * 8;
  XK_CUDA(cudaMemcpyAsync(h->Ce, C, cb, cudaMemcpyHostToDevice, h->stream));
  int rc = enqueue_energy(h);
  if (rc != XK_OK) return rc;
  XK_CUDA(cudaMemcpyAsync(Ex, h->Ce + (size_t)h->N * h->n, 8, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaStreamSynchronize(h->stream));
  {
    cudaError_t e = cudaSuccess;
    const int st = take_status(h, h->stream, &e);
    if (e != cudaSuccess) return cuda_fail(e, "xk_energy status");
    if (st != 0)
      return fail(XK_ETIMEDOUT, "xk_energy: a bounded wait inside a kernel gave up (code " +
                                    std::to_string(st) + ")");
  }
  return XK_OK;
}

int xk_energy_device(xk_handle* h, const double* C_dev, double* Ex_dev, void* stream) {
  if (!h || !C_dev || !Ex_dev) return fail(XK_EINVAL, "xk_energy_device: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev;
  XK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  XK_CUDA(cudaEventRecord(ev, us));
  XK_CUDA(cudaStreamWaitEvent(h->stream, ev, 0));
  XK_CUDA(cudaMemcpyAsync(h->Ce, C_dev, (size_t)h->N * h->n * 8, cudaMemcpyDeviceToDevice, h->stream));
  int rc = enqueue_energy(h);
  if (rc != XK_OK) { cudaEventDestroy(ev); return rc; }
  XK_CUDA(cudaMemcpyAsync(Ex_dev, h->Ce + (size_t)h->N * h->n, 8, cudaMemcpyDeviceToDevice, h->stream));
  XK_CUDA(cudaEventRecord(ev, h->stream));
  XK_CUDA(cudaStreamWaitEvent(us, ev, 0));
  cudaEventDestroy(ev);
  return XK_OK;
}

int xk_ace(xk_handle* h, double* Kij_out, double* xi_out, double* sign_out, int* branch) {
  if (!h || !Kij_out || !xi_out) return fail(XK_EINVAL, "xk_ace: NULL argument");
  if (h->ga != h->Naux)
    return fail(XK_EINVAL, "xk_ace: a shard's K is a partial sum; factor the summed K");
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->has_build) return fail(XK_EINVAL, "xk_ace: no completed build on this handle");
  DeviceGuard g(h->device);
  cudaStream_t s = h->stream;
  const int N = h->N, n = h->n;
  xk::DGemm kij{n, n, N, h->C, n, true, h->K, n, false, h->Kij, n, 1.0, nullptr, 0, 0, h->work};
  XK_CUDA(xk::dgemm(kij, s));
  XK_CUDA(xk::symmetrize_f64(h->Kij, n, s));
  XK_CUDA(cudaMemcpyAsync(h->Lf, h->Kij, (size_t)n * n * 8, cudaMemcpyDeviceToDevice, s));
  XK_CUDA(xk::cholesky_f64(h->Lf, n, h->status, s));
  int st = 0;
  XK_CUDA(cudaMemcpyAsync(&st, h->status, 4, cudaMemcpyDeviceToHost, s));
  XK_CUDA(cudaStreamSynchronize(s));
  int br = 0;
  std::vector<double> sg(n, 1.0);
  if (st == 0) {
    XK_CUDA(xk::trsm_right_lt_f64(h->Lf, n, h->K, N, h->xi, s));
  } else {
    br = 1;
    XK_CUDA(cudaMemcpyAsync(h->Lf, h->Kij, (size_t)n * n * 8, cudaMemcpyDeviceToDevice, s));
    XK_CUDA(xk::jacobi_eig_f64(h->Lf, h->U, n, 60, h->status + 1, s));
    xk::DGemm ku{N, n, n, h->K, n, false, h->U, n, false, h->Y, n, 1.0, nullptr, 0, 0, h->work};
    XK_CUDA(xk::dgemm(ku, s));
    XK_CUDA(xk::scale_eigcols_f64(h->Lf, n, h->Y, N, 1e-12, h->xi, h->sgn, s));
    XK_CUDA(cudaMemcpyAsync(sg.data(), h->sgn, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  }
  XK_CUDA(cudaMemcpyAsync(Kij_out, h->Kij, (size_t)n * n * 8, cudaMemcpyDeviceToHost, s));
  XK_CUDA(cudaMemcpyAsync(xi_out, h->xi, (size_t)N * n * 8, cudaMemcpyDeviceToHost, s));
  XK_CUDA(cudaStreamSynchronize(s));
  if (sign_out) std::memcpy(sign_out, sg.data(), (size_t)n * 8);
  if (branch) *branch = br;
  return XK_OK;
}

int xk_submit(xk_handle* h, const double* C, double deadline_ms, xk_ticket* t) {
  if (!h || !C || !t) return fail(XK_EINVAL, "xk_submit: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  int k = -1;
  for (int i = 0; i < kSlots; ++i) {
    Slot& s = h->slots[i];
    if (s.state == 2 && cudaEventQuery(s.done) == cudaSuccess) s.state = 0;
    if (s.state == 0 && k < 0) k = i;
  }
  if (k < 0) return fail(XK_EBUSY, "xk_submit: every slot of the handle is in flight");
  Slot& s = h->slots[k];
  const size_t kb = (size_t)h->N * h->n * 8;
  std::memcpy(s.C, C, kb);
  XK_CUDA(cudaMemcpyAsync(h->C, s.C, kb, cudaMemcpyHostToDevice, h->stream));
  int rc = enqueue_build(h);
  if (rc != XK_OK) return rc;
  XK_CUDA(cudaMemcpyAsync(s.K, h->K, kb, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaMemcpyAsync(s.Ex, h->Ex, 16, cudaMemcpyDeviceToHost, h->stream));
  // this build's status word, taken and cleared in stream order: every slot
  // reports the kernels of its own build
  s.st[0] = 0;
  if (h->mixed) {
    int* dev = xk::mixed_status_ptr(h->mixed);
    XK_CUDA(cudaMemcpyAsync(s.st, dev, 16, cudaMemcpyDeviceToHost, h->stream));
    XK_CUDA(cudaMemsetAsync(dev, 0, 16, h->stream));
  }
  XK_CUDA(cudaEventRecord(s.done, h->stream));
  h->has_build = true;
  s.state = 1;
  s.has_deadline = deadline_ms > 0;
  if (s.has_deadline)
    s.deadline = std::chrono::steady_clock::now() +
                 std::chrono::microseconds((long long)(deadline_ms * 1000.0));
  std::lock_guard<std::mutex> tl(g_tickets_mu);
  s.ticket = g_next_ticket++;
  g_tickets[s.ticket] = {h, k};
  *t = s.ticket;
  return XK_OK;
}

int xk_poll(xk_ticket t, double* K_out, double* Ex, double* err_est) {
  if (!K_out || !Ex) return fail(XK_EINVAL, "xk_poll: NULL argument");
  xk_handle* h = nullptr;
  int k = -1;
  {
    std::lock_guard<std::mutex> tl(g_tickets_mu);
    auto it = g_tickets.find(t);
    if (it == g_tickets.end()) return fail(XK_EINVAL, "xk_poll: unknown ticket");
    h = it->second.first;
    k = it->second.second;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  Slot& s = h->slots[k];
  cudaError_t q = cudaEventQuery(s.done);
  auto consume = [&]() {
    std::lock_guard<std::mutex> tl(g_tickets_mu);
    g_tickets.erase(t);
  };
  if (q == cudaErrorNotReady) {
    if (s.has_deadline && std::chrono::steady_clock::now() > s.deadline) {
      s.state = 2;
      consume();
      return fail(XK_ETIMEDOUT, "xk_poll: ticket deadline expired");
    }
    return XK_PENDING;
  }
  if (q != cudaSuccess) {
    s.state = 0;
    consume();
    return cuda_fail(q, "xk_poll");
  }
  const size_t kb = (size_t)h->N * h->n * 8;
  if (s.st[0] != 0) {
    const int st = s.st[0];
    s.state = 0;
    consume();
    return fail(XK_ETIMEDOUT, "xk_poll: a bounded wait inside a kernel gave up (code " +
                                  std::to_string(st) + ")");
  }
  std::memcpy(K_out, s.K, kb);
  *Ex = *s.Ex;
  if (err_est) *err_est = std::fabs(s.Ex[0] - s.Ex[1]);
  s.state = 0;
  consume();
  return XK_OK;
}

int xk_timing_enable(xk_handle* h, int enable) {
  if (!h) return fail(XK_EINVAL, "xk_timing_enable: NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  XK_CUDA(cudaStreamSynchronize(h->stream));
  fold_marks(h);
  for (int i = 0; i < XK_NSTEPS; ++i) {
    h->step_ms[i] = 0.0;
    h->step_builds[i] = 0;
  }
  h->timing = enable != 0;
  return XK_OK;
}

int xk_timing_read(xk_handle* h, int step, double* ms, uint64_t* builds) {
  if (!h || !ms || step < 0 || step >= XK_NSTEPS)
    return fail(XK_EINVAL, "xk_timing_read: bad argument");
  std::lock_guard<std::mutex> lk(h->mu);
  DeviceGuard g(h->device);
  XK_CUDA(cudaStreamSynchronize(h->stream));
  fold_marks(h);
  *ms = h->step_ms[step];
  if (builds) *builds = h->step_builds[step];
  return XK_OK;
}

int xk_exchange_energy_noalloc(const double* K_dev, const double* C_dev, int64_t count,
                               double* Ex_dev, void* stream) {
  if (!K_dev || !C_dev || !Ex_dev)
    return fail(XK_EINVAL, "xk_exchange_energy_noalloc: NULL pointer");
  if (count < 0 || count > xk::noalloc_max_count())
    return fail(XK_EINVAL, "xk_exchange_energy_noalloc: count " + std::to_string(count) +
                               " is outside [0, " + std::to_string(xk::noalloc_max_count()) + "]");
  cudaError_t e = xk::exchange_energy_noalloc(K_dev, C_dev, count, Ex_dev,
                                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "xk_exchange_energy_noalloc");
  return XK_OK;
}

int xk_release(xk_handle* h) {
  if (!h) return fail(XK_EINVAL, "xk_release: NULL handle");
  {
    // after any call that holds the handle (lock order: handle, then tickets)
    std::lock_guard<std::mutex> lk(h->mu);
    std::lock_guard<std::mutex> tl(g_tickets_mu);
    for (auto it = g_tickets.begin(); it != g_tickets.end();)
      it = (it->second.first == h) ? g_tickets.erase(it) : std::next(it);
  }
  free_handle(h);
  return XK_OK;
}

int xk_error_estimate(xk_handle* h, double* est) {
  if (!h || !est) return fail(XK_EINVAL, "xk_error_estimate: NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->has_build) return fail(XK_EINVAL, "xk_error_estimate: no build on this handle yet");
  DeviceGuard g(h->device);
  double e2[2] = {0.0, 0.0};
  XK_CUDA(cudaMemcpyAsync(e2, h->Ex, 16, cudaMemcpyDeviceToHost, h->stream));
  XK_CUDA(cudaStreamSynchronize(h->stream));
  *est = std::fabs(e2[0] - e2[1]);
  return XK_OK;
}

int xk_autotune_info(xk_handle* h, int32_t* info, double* ms) {
  if (!h || !info || !ms) return fail(XK_EINVAL, "xk_autotune_info: NULL argument");
  if (!h->mixed) return fail(XK_EINVAL, "xk_autotune_info: not an XK_F16X3 handle");
  std::lock_guard<std::mutex> lk(h->mu);
  int in[2] = {0, 0};
  double t[3] = {0.0, 0.0, 0.0};
  xk::mixed_autotune_info(h->mixed, in, t);
  info[0] = in[0];
  info[1] = in[1];
  ms[0] = t[0]; ms[1] = t[1]; ms[2] = t[2];
  return XK_OK;
}

int xk_set_wait_limit(xk_handle* h, int64_t cycles) {
  if (!h || cycles < 0) return fail(XK_EINVAL, "xk_set_wait_limit: NULL handle or negative limit");
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->mixed) xk::mixed_set_wait_limit(h->mixed, (long long)cycles);
  drop_graph(h);  // its kernels hold the old limit
  return XK_OK;
}

// ---------------------------------------------------------------- batches

struct xk_batch {
  std::vector<xk_handle*> hs;
  int device = 0;
  cudaStream_t stream = nullptr;
  // capture-time fork/join: the members' orbital and line steps run on up to
  // kBatchSide streams side by side (their small kernels overlap), the
  // grouped pair launch on `stream` between them
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> evs;  // 2 forks, then 2 x side.size() joins
  xk::PairGroup* group = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;  // kernels in one replay of the graph
};

int xk_batch_create(xk_handle* const* handles, int count, xk_batch** out) {
  if (!out) return fail(XK_EINVAL, "xk_batch_create: out is NULL");
  *out = nullptr;
  if (!handles || count <= 0) return fail(XK_EINVAL, "xk_batch_create: no handles");
  std::vector<xk_handle*> hs(handles, handles + count);
  for (xk_handle* h : hs) {
    if (!h) return fail(XK_EINVAL, "xk_batch_create: NULL handle");
    if (h->mode != XK_F16X3 || !h->mixed)
      return fail(XK_EINVAL, "xk_batch_create: every handle must use XK_F16X3");
    if (h->device != hs[0]->device)
      return fail(XK_EINVAL, "xk_batch_create: handles on different devices");
  }
  {
    std::vector<xk_handle*> t = hs;
    std::sort(t.begin(), t.end());
    if (std::adjacent_find(t.begin(), t.end()) != t.end())
      return fail(XK_EINVAL, "xk_batch_create: a handle appears twice");
  }
  DeviceGuard g(hs[0]->device);
  xk_batch* b = new xk_batch();
  b->hs = hs;
  b->device = hs[0]->device;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  constexpr int kBatchSide = 8;
  const int nside = std::min(count, kBatchSide);
  for (int k = 0; k < nside && e == cudaSuccess; ++k) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->side.push_back(st);
  }
  for (int k = 0; k < 2 + 2 * nside && e == cudaSuccess; ++k) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->evs.push_back(ev);
  }
  std::vector<xk::MixedState*> ms;
  for (xk_handle* h : hs) ms.push_back(h->mixed);
  if (e == cudaSuccess) e = xk::mixed_group_create(ms.data(), count, &b->group);
  if (e != cudaSuccess) {
    for (cudaEvent_t ev : b->evs) cudaEventDestroy(ev);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return cuda_fail(e, "xk_batch_create");
  }
  *out = b;
  return XK_OK;
}

int xk_batch_build(xk_batch* b, const double* const* C, double* const* K_out, double* Ex_out) {
  if (!b || !C || !K_out || !Ex_out) return fail(XK_EINVAL, "xk_batch_build: NULL argument");
  const size_t count = b->hs.size();
  for (size_t i = 0; i < count; ++i)
    if (!C[i] || !K_out[i]) return fail(XK_EINVAL, "xk_batch_build: NULL coefficient or K pointer");
  // lock the members in address order (no lock-order cycles with other batches)
  std::vector<xk_handle*> order = b->hs;
  std::sort(order.begin(), order.end());
  std::vector<std::unique_lock<std::mutex>> locks;
  for (xk_handle* h : order) locks.emplace_back(h->mu);
  DeviceGuard g(b->device);
  // after any work still queued on the members' own streams, then the inputs
  for (xk_handle* h : b->hs) {
    cudaEvent_t ev;
    XK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    XK_CUDA(cudaEventRecord(ev, h->stream));
    XK_CUDA(cudaStreamWaitEvent(b->stream, ev, 0));
    cudaEventDestroy(ev);
  }
  for (size_t i = 0; i < count; ++i) {
    xk_handle* h = b->hs[i];
    XK_CUDA(cudaMemcpyAsync(h->C, C[i], (size_t)h->N * h->n * 8, cudaMemcpyHostToDevice, b->stream));
  }
  if (!b->exec) {
    // the whole batch, device work only, captured once into a graph: the
    // orbitals of every member, one grouped pair launch, the line steps
    const uint64_t l0 = xk::g_launches.load();
    XK_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    xk::StepHook none{nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    const size_t ns = b->side.size();
    // the side streams start after `stream` (fork) and `stream` continues
    // after all of them (join)
    auto fork = [&](int f) {
      if (e == cudaSuccess) e = cudaEventRecord(b->evs[f], b->stream);
      for (size_t k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->evs[f], 0);
    };
    auto join = [&](int f) {
      for (size_t k = 0; k < ns && e == cudaSuccess; ++k) {
        cudaEvent_t ev = b->evs[2 + f * ns + k];
        e = cudaEventRecord(ev, b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
      }
    };
    fork(0);
    for (size_t i = 0; i < b->hs.size(); ++i)
      if (e == cudaSuccess) e = xk::mixed_enqueue_pre(b->hs[i]->mixed, b->hs[i]->C, b->side[i % ns], none);
    join(0);
    if (e == cudaSuccess) e = xk::mixed_group_enqueue_pair(b->group, b->stream);
    fork(1);
    for (size_t i = 0; i < b->hs.size(); ++i)
      if (e == cudaSuccess)
        e = xk::mixed_enqueue_post(b->hs[i]->mixed, b->hs[i]->K, b->hs[i]->Ex, b->side[i % ns], none);
    join(1);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      b->exec = nullptr;
      return cuda_fail(e, "xk_batch_build: graph capture");
    }
    b->graph = graph;
    b->launches = xk::g_launches.load() - l0;
    xk::g_launches.fetch_sub(b->launches);  // counted again per replay below
  }
  XK_CUDA(cudaGraphLaunch(b->exec, b->stream));
  xk::g_launches.fetch_add(b->launches);
  for (size_t i = 0; i < count; ++i) {
    xk_handle* h = b->hs[i];
    XK_CUDA(cudaMemcpyAsync(K_out[i], h->K, (size_t)h->N * h->n * 8, cudaMemcpyDeviceToHost, b->stream));
    XK_CUDA(cudaMemcpyAsync(Ex_out + i, h->Ex, 8, cudaMemcpyDeviceToHost, b->stream));
  }
  XK_CUDA(cudaStreamSynchronize(b->stream));
  // every member's status word, each read and cleared before returning
  int first = 0;
  for (xk_handle* h : b->hs) {
    h->has_build = true;
    cudaError_t e = cudaSuccess;
    const int st = take_status(h, b->stream, &e);
    if (e != cudaSuccess) return cuda_fail(e, "xk_batch_build status");
    if (st != 0 && first == 0) first = st;
  }
  if (first != 0)
    return fail(XK_ETIMEDOUT, "xk_batch_build: a bounded wait inside a kernel gave up (code " +
                                  std::to_string(first) + ")");
  return XK_OK;
}

int xk_batch_release(xk_batch* b) {
  if (!b) return fail(XK_EINVAL, "xk_batch_release: NULL batch");
  DeviceGuard g(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  xk::mixed_group_destroy(b->group);
  for (cudaEvent_t ev : b->evs) cudaEventDestroy(ev);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return XK_OK;
}

}  // extern "C"
