// C ABI of the all-shift NGF similarity library: handle management, host-side
// rotation matrices, workspace sizing and the per-batch launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/cs_ngf.h"
#include "handle.h"
#include "kernels.cuh"

using namespace csngf;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace csngf {
// lets other translation units of the library report through cs_ngf_last_error
void set_last_error(const std::string& msg) { g_last_error = msg; }
namespace detail {
cs_ngf_status fail(cs_ngf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
}  // namespace detail
}  // namespace csngf

using csngf::detail::fail;

namespace {

#define CS_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? CS_NGF_ENOMEM : CS_NGF_ECUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

constexpr int kPads[] = {16, 32, 40, 64, 80, 100, 128, 160, 192, 200, 216, 256, 320, 360, 400, 512};

bool pad_supported(int p) {
  for (int v : kPads)
    if (v == p) return true;
  return false;
}

int auto_pad(int n) {
  for (int v : kPads)
    if (v >= 2 * n - 1) return v;
  return 0;
}

// Hamilton unit quaternion (w, x, y, z) -> row-major matrix on (x, y, z), FP64,
// entries within 1e-9 of -1, 0, 1 snapped (exact identity and quarter turns).
void quat_to_rotmat(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  const double s = std::sqrt(w * w + x * x + y * y + z * z);
  w = w / s;
  x = x / s;
  y = y / s;
  z = z / s;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
  const double targets[3] = {-1.0, 0.0, 1.0};
  for (double tgt : targets)
    for (int i = 0; i < 9; ++i)
      if (std::fabs(R[i] - tgt) <= 1e-9) R[i] = tgt;
}

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T));
}

}  // namespace


namespace {

std::atomic<long long> g_launches{0};

// brackets one kernel launch: counts it and, when profiling, times it with
// events on the launching stream
struct Stage {
  cs_ngf_fixed* f;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Stage(cs_ngf_fixed* f_, int s_, cudaStream_t st_) : f(f_), stage(s_), st(st_) {
    if (f->profiling && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  ~Stage() {
    if (!f->capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (a) {
      cudaEvent_t b = nullptr;
      if (cudaEventCreate(&b) == cudaSuccess) {
        cudaEventRecord(b, st);
        f->spans.push_back({stage, a, b});
      } else {
        cudaEventDestroy(a);
      }
    }
  }
};

// -------------------------------------------------------------- dispatch
#define CS_DISPATCH(P, CALL)                                                           \
  switch (P) {                                                                          \
    case 16: { constexpr int PP = 16; CALL; } break;                                    \
    case 32: { constexpr int PP = 32; CALL; } break;                                    \
    case 40: { constexpr int PP = 40; CALL; } break;                                    \
    case 64: { constexpr int PP = 64; CALL; } break;                                    \
    case 80: { constexpr int PP = 80; CALL; } break;                                    \
    case 100: { constexpr int PP = 100; CALL; } break;                                  \
    case 128: { constexpr int PP = 128; CALL; } break;                                  \
    case 160: { constexpr int PP = 160; CALL; } break;                                  \
    case 192: { constexpr int PP = 192; CALL; } break;                                  \
    case 200: { constexpr int PP = 200; CALL; } break;                                  \
    case 216: { constexpr int PP = 216; CALL; } break;                                  \
    case 256: { constexpr int PP = 256; CALL; } break;                                  \
    case 320: { constexpr int PP = 320; CALL; } break;                                  \
    case 360: { constexpr int PP = 360; CALL; } break;                                  \
    case 400: { constexpr int PP = 400; CALL; } break;                                  \
    case 512: { constexpr int PP = 512; CALL; } break;                                  \
    default: break;                                                                     \
  }

cs_ngf_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CS_NGF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return CS_NGF_OK;
}

// ECUDA (once) if a tensor-core pass of this handle stopped on its bounded
// wait since the last check; `st` has been synchronised by the caller
cs_ngf_status tc_status(cs_ngf_fixed* f, cudaStream_t st) {
  if (!f->tc_err) return CS_NGF_OK;
  int flag = 0;
  CS_CUDA(cudaMemcpyAsync(&flag, f->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaStreamSynchronize(st));
  if (!flag) return CS_NGF_OK;
  CS_CUDA(cudaMemsetAsync(f->tc_err, 0, sizeof(int), st));
  return fail(CS_NGF_ECUDA, "a tensor-core z pass timed out waiting for its MMAs; its results are invalid");
}

void free_handle(cs_ngf_fixed* f) {
  if (!f) return;
  DeviceGuard guard(f->device);
  cudaFree(f->UV);
  cudaFree(f->Bh);
  cudaFree(f->Mh);
  cudaFree(f->BQ);
  cudaFree(f->C8);
  cudaFree(f->F02);
  cudaFree(f->F13);
  cudaFree(f->msum);
  cudaFree(f->margA);
  cudaFree(f->margB);
  cudaFree(f->bounds);
  cudaFree(f->thr);
  cudaFree(f->keys);
  cudaFree(f->tc_err);
  cudaFree(f->zx);
  for (int a = 0; a < 3; ++a) {
    bool dup = false;
    for (int b = 0; b < a; ++b) dup |= (f->tw[b] == f->tw[a]);
    if (!dup) cudaFree(f->tw[a]);
  }
  if (f->rot_ev) cudaEventSynchronize(f->rot_ev);
  if (f->order_ev) cudaEventDestroy(f->order_ev);
  for (auto& sp : f->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
  if (f->gexec) cudaGraphExecDestroy(f->gexec);
  for (auto& gs : f->graphs) cudaGraphExecDestroy(gs.exec);
  cudaFree(f->allb);
  cudaFreeHost(f->allb_h);
  cudaFree(f->perm_d);
  cudaFree(f->perm_score);
  cudaFree(f->perm_shift);
  cudaFree(f->rot_slot);
  cudaFree(f->slot_score);
  cudaFree(f->slot_shift);
  cudaFreeHost(f->rot_h);
  cudaFree(f->rot_d);
  if (f->rot_ev) cudaEventDestroy(f->rot_ev);
  cudaFree(f->stage_B);
  cudaFree(f->stage_M);
  cudaFree(f->res_score);
  cudaFree(f->res_shift);
  cudaFree(f->A_keep);
  cudaFree(f->MA_keep);
  delete f;
}

// twiddle table exp(-2 pi i m / P), m < P, into dst (at least P entries);
// synchronous, so no kernel may still read dst
cs_ngf_status fill_twiddles(int P, float2* dst) {
  std::vector<float2> h(P);
  for (int m = 0; m < P; ++m) {
    h[m].x = (float)ctw::cos2pi(m, P);
    h[m].y = (float)(-ctw::sin2pi(m, P));
  }
  CS_CUDA(cudaMemcpy(dst, h.data(), sizeof(float2) * P, cudaMemcpyHostToDevice));
  return CS_NGF_OK;
}

// upload R rotation matrices (host FP64 quaternions) to f->rot_d
cs_ngf_status upload_rotations(cs_ngf_fixed* f, const double* quats, int R, cudaStream_t st) {
  if (!quats) return fail(CS_NGF_EINVAL, "quats is NULL");
  for (int r = 0; r < R; ++r) {
    const double* q = quats + 4 * r;
    const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(std::fabs(n - 1.0) <= 1e-3))
      return fail(CS_NGF_EINVAL, "quaternion " + std::to_string(r) + " is not unit (norm " +
                                     std::to_string(n) + ")");
  }
  if (f->rot_ev) CS_CUDA(cudaEventSynchronize(f->rot_ev));   // previous upload has left rot_h
  if (R > f->rot_cap) {
    if (f->rot_ev) CS_CUDA(cudaDeviceSynchronize());          // rot_d may still be read
    cudaFreeHost(f->rot_h);
    cudaFree(f->rot_d);
    f->rot_h = nullptr;
    f->rot_d = nullptr;
    f->rot_cap = 0;
    const int cap = std::max(R, 64);
    CS_CUDA(cudaMallocHost((void**)&f->rot_h, sizeof(RotMat) * cap));
    CS_CUDA(dalloc(&f->rot_d, (size_t)cap));
    f->rot_cap = cap;
  }
  if (!f->rot_ev) CS_CUDA(cudaEventCreateWithFlags(&f->rot_ev, cudaEventDisableTiming));
  for (int r = 0; r < R; ++r) {
    double Rm[9];
    quat_to_rotmat(quats + 4 * r, Rm);
    for (int i = 0; i < 9; ++i) f->rot_h[r].m[i] = (float)Rm[i];
  }
  CS_CUDA(cudaMemcpyAsync(f->rot_d, f->rot_h, sizeof(RotMat) * R, cudaMemcpyHostToDevice, st));
  CS_CUDA(cudaEventRecord(f->rot_ev, st));
  return CS_NGF_OK;
}

// ------------------------------------------------------------ autotuning
// Process-wide choice of radix split per FFT pass, keyed by the pass, its
// length, whether its input fills at most half the length, and the storage
// form of the channel fields; with the best time of each variant.
struct TuneKey {
  int pass, P, half, store;
  bool operator<(const TuneKey& o) const {
    return std::tie(pass, P, half, store) < std::tie(o.pass, o.P, o.half, o.store);
  }
};
struct TuneVal { int variant; float ms[2]; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

constexpr int kPasses = 5;   // fwd_x, fwd_y, zmac, inv_y, inv_x

// (N1, N2) of split variant v of length P; (0, 0) if P has no such variant
template <int P>
void split_into(int v, int32_t* n1, int32_t* n2) {
  *n1 = *n2 = 0;
  if constexpr (has_alt_split(P)) {
    if (v == 1) {
      *n1 = SplitV<P, 1>::N1;
      *n2 = SplitV<P, 1>::N2;
    }
  }
  if (v == 0) {
    *n1 = SplitV<P, 0>::N1;
    *n2 = SplitV<P, 0>::N2;
  }
}
void split_of(int P, int v, int32_t* n1, int32_t* n2) {
  *n1 = *n2 = 0;
  CS_DISPATCH(P, split_into<PP>(v, n1, n2));
}

// the key of pass k at the handle's lengths in use
TuneKey tune_key(const cs_ngf_fixed* f, int k) {
  const Geo& g = f->g;
  switch (k) {
    case 0: return {0, g.Px, 2 * g.nx <= g.Px, g.store};
    case 1: return {1, g.Py, 2 * g.ny <= g.Py, g.store};
    case 2: return {2, g.Pz, 2 * g.nz <= g.Pz, g.store};
    case 3: return {3, g.Py, 0, 0};
    default: return {4, g.Px, 0, 0};
  }
}

// the variants the handle uses at its lengths in use: the table's choices
// when autotuning, the alternative wherever there is one in mode 2, else the
// built-in splits
void resolve_variants(cs_ngf_fixed* f) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int k = 0; k < kPasses; ++k) {
    f->vars[k] = 0;
    if (f->autotune == 2) {
      f->vars[k] = has_alt_split(tune_key(f, k).P) ? 1 : 0;
      continue;
    }
    if (f->autotune != 1) continue;
    auto it = g_tune.find(tune_key(f, k));
    if (it != g_tune.end()) f->vars[k] = it->second.variant;
  }
}

// some pass at the lengths in use has two splits and no choice yet
bool needs_tuning(const cs_ngf_fixed* f) {
  if (f->autotune != 1) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int k = 0; k < kPasses; ++k) {
    const TuneKey key = tune_key(f, k);
    if (has_alt_split(key.P) && g_tune.find(key) == g_tune.end()) return true;
  }
  return false;
}

// launch FFT pass k of nb volumes with split variant v
void launch_pass(cs_ngf_fixed* f, int k, int v, int nb, float* map, cudaStream_t st) {
  const Geo& g = f->g;
  switch (k) {
    case 0: CS_DISPATCH(g.Px, launch_fwd_x<PP>(f->Bh, f->Mh, f->F02, f->tw[2], g, nb, st, v)); break;
    case 1: CS_DISPATCH(g.Py, launch_fwd_y<PP>(f->F02, f->F13, f->tw[1], g, nb, st, v)); break;
    case 2: CS_DISPATCH(g.Pz, launch_zmac<PP>(f->F13, f->UV, f->F02, f->tw[0], g, nb, f->bounds, st, v)); break;
    case 3: CS_DISPATCH(g.Py, launch_inv_y<PP>(f->F02, f->F13, f->tw[1], g, nb, f->bounds, st, v)); break;
    default: CS_DISPATCH(g.Px, launch_inv_x<PP>(f->F13, f->thr, f->keys, map, f->tw[2], g, nb, f->bounds, st, v)); break;
  }
}

const char* const kPassName[kPasses] = {"fwd_x", "fwd_y", "zmac", "inv_y", "inv_x"};

// Time both variants of pass k (best of two runs each, on the inputs the
// previous passes left), record the faster and run it once more, so that
// its output is what the next pass reads.  A pass is repeatable: it reads
// buffers it does not write, except the x inverse's per-rotation maxima,
// which are cleared before the final run.
cs_ngf_status tune_pass(cs_ngf_fixed* f, int k, int nb, cudaStream_t st) {
  const TuneKey key = tune_key(f, k);
  float best[2] = {0.0f, 0.0f};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CS_CUDA(cudaEventCreate(&e0));
  CS_CUDA(cudaEventCreate(&e1));
  cs_ngf_status s = CS_NGF_OK;
  for (int v = 0; v < 2 && !s; ++v)
    for (int rep = 0; rep < 2 && !s; ++rep) {
      cudaEventRecord(e0, st);
      { Stage sp(f, 1 + k, st); launch_pass(f, k, v, nb, nullptr, st); }
      cudaEventRecord(e1, st);
      if ((s = check_launch(kPassName[k]))) break;
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        s = fail(CS_NGF_ECUDA, "autotune timing failed");
      if (rep == 0 || ms < best[v]) best[v] = ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  const int choice = best[1] < best[0] ? 1 : 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {choice, {best[0], best[1]}};
  }
  f->vars[k] = choice;
  if (k == 4) CS_CUDA(cudaMemsetAsync(f->keys, 0, sizeof(unsigned long long) * nb, st));
  { Stage sp(f, 1 + k, st); launch_pass(f, k, choice, nb, nullptr, st); }
  return check_launch(kPassName[k]);
}

// the FFT passes for nb volumes already resampled into f->Bh / f->Mh; with
// tune, passes whose two splits have no choice yet are timed first
cs_ngf_status run_transforms(cs_ngf_fixed* f, int nb, float* map, cudaStream_t st, bool tune = false) {
  for (int k = 0; k < kPasses; ++k) {
    if (tune && !map) {
      const TuneKey key = tune_key(f, k);
      bool untuned = false;
      if (has_alt_split(key.P)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        untuned = g_tune.find(key) == g_tune.end();
      }
      if (untuned) {
        if (cs_ngf_status s = tune_pass(f, k, nb, st)) return s;
        continue;
      }
    }
    { Stage sp(f, 1 + k, st); launch_pass(f, k, f->vars[k], nb, map, st); }
    if (cs_ngf_status s = check_launch(kPassName[k])) return s;
  }
  return CS_NGF_OK;
}

// (B, M_B) -> f->BQ, f->C8, shared by every rotation of the call
cs_ngf_status pack_floating(cs_ngf_fixed* f, const float* B, const uint8_t* MB, cudaStream_t st) {
  { Stage sp(f, 0, st); k_pack_floating<<<512, 256, 0, st>>>(B, MB, f->g, f->BQ, f->C8); }
  return check_launch("pack");
}

// score nb rotations whose matrices are at rot (device), with the floating
// volume already packed in f->BQ, f->C8; results to out_score[nb], out_shift[nb][3]
cs_ngf_status score_batch_ptrs(cs_ngf_fixed* f, const RotMat* rot, int nb, float* out_score,
                               int32_t* out_shift, float* map, cudaStream_t st, bool tune = false) {
  const Geo& g = f->g;
  const size_t nmarg = (size_t)g.nz + g.ny + g.nx;
  CS_CUDA(cudaMemsetAsync(f->msum, 0, sizeof(int) * nb, st));
  CS_CUDA(cudaMemsetAsync(f->keys, 0, sizeof(unsigned long long) * nb, st));
  CS_CUDA(cudaMemsetAsync(f->margB, 0, sizeof(int) * nmarg * nb, st));
  {
    Stage sp(f, 0, st);
    k_resample<<<resample_grid(g, nb), 128, 0, st>>>(f->BQ, f->C8, rot, g, f->Bh, f->Mh, f->msum, f->margB);
  }
  if (cs_ngf_status s = check_launch("resample")) return s;
  const double pvol = (double)g.Px * (double)g.Py * (double)g.Pz;
  {
    Stage sp(f, 7, st);
    k_thresholds<<<(nb + 127) / 128, 128, 0, st>>>(f->msum, f->sumA, f->gamma, pvol, nb, f->thr);
  }
  if (cs_ngf_status s = check_launch("thresholds")) return s;
  {
    Stage sp(f, 7, st);
    k_shift_bounds<<<dim3((unsigned)nb, 3u), 512, 0, st>>>(f->margA, f->margB, f->msum, f->sumA,
                                                           f->gamma, g, f->bounds);
  }
  if (cs_ngf_status s = check_launch("shift bounds")) return s;
  if (map) {
    Stage sp(f, 7, st);
    k_fill<<<256, 256, 0, st>>>(map, (long long)g.vz * g.vy * g.vx, -INFINITY);
  }
  if (cs_ngf_status s = run_transforms(f, nb, map, st, tune)) return s;
  {
    Stage sp(f, 7, st);
    k_finalize<<<(nb + 127) / 128, 128, 0, st>>>(f->keys, nb, g, out_score, out_shift);
  }
  return check_launch("finalize");
}

constexpr int kKernelsPerBatch = 9;   // resample, thresholds, bounds, 5 passes, finalize

cs_ngf_status score_batch(cs_ngf_fixed* f, int r0, int nb, float* best_score, int32_t* best_shift,
                          float* map, cudaStream_t st, bool tune = false) {
  return score_batch_ptrs(f, f->rot_d + r0, nb, best_score + r0, best_shift + 3 * (size_t)r0, map, st,
                          tune);
}

// capture the full-batch launch sequence once (on a private stream; the
// graph is then replayed on the caller's stream)
cs_ngf_status ensure_graph(cs_ngf_fixed* f) {
  if (f->gexec && !std::equal(f->vars, f->vars + kPasses, f->gexec_vars)) {   // captured with other splits
    cudaGraphExecDestroy(f->gexec);
    f->gexec = nullptr;
  }
  if (f->gexec) return CS_NGF_OK;
  std::copy(f->vars, f->vars + kPasses, f->gexec_vars);
  if (!f->rot_slot) {
    CS_CUDA(dalloc(&f->rot_slot, (size_t)f->batch));
    CS_CUDA(dalloc(&f->slot_score, (size_t)f->batch));
    CS_CUDA(dalloc(&f->slot_shift, (size_t)f->batch * 3));
  }
  cudaStream_t cs = nullptr;
  CS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cs_ngf_status st = CS_NGF_OK;
  if (e == cudaSuccess) {
    f->capturing = true;
    st = score_batch_ptrs(f, f->rot_slot, f->batch, f->slot_score, f->slot_shift, nullptr, cs);
    f->capturing = false;
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess && st == CS_NGF_OK) e = cudaGraphInstantiate(&f->gexec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (st != CS_NGF_OK) return st;
  if (e != cudaSuccess) {
    f->gexec = nullptr;
    return fail(CS_NGF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  return CS_NGF_OK;
}

// Section 3.1 A side: NGF channels of A times M_A, forward FFTs, weights -> f->UV
cs_ngf_status run_fixed(cs_ngf_fixed* f, const float* A, const uint8_t* MA, cudaStream_t st) {
  Geo g = f->g;
  g.store = kStoreF32;            // the fixed spectra are always computed in FP32
  for (int j = 0; j < 4; ++j) g.scale0[j] = g.scale1[j] = 1.0f;
  { Stage sp(f, 6, st); k_copy_in<<<1024, 256, 0, st>>>(A, MA, g.nvox, f->Bh, f->Mh); }
  if (cs_ngf_status s = check_launch("copy_in")) return s;
  CS_CUDA(cudaMemsetAsync(f->msum, 0, sizeof(int), st));
  { Stage sp(f, 6, st); k_mask_sum<<<1024, 256, 0, st>>>(f->Mh, g.nvox, f->msum); }
  if (cs_ngf_status s = check_launch("mask_sum")) return s;
  CS_CUDA(cudaMemsetAsync(f->margA, 0, sizeof(int) * ((size_t)g.nz + g.ny + g.nx), st));
  { Stage sp(f, 6, st); k_marginals<<<1024, 256, 0, st>>>(f->Mh, g, f->margA); }
  if (cs_ngf_status s = check_launch("marginals")) return s;
  { Stage sp(f, 6, st); CS_DISPATCH(g.Px, launch_fwd_x<PP>(f->Bh, f->Mh, f->F02, f->tw[2], g, 1, st)); }
  if (cs_ngf_status s = check_launch("fwd_x (fixed)")) return s;
  { Stage sp(f, 6, st); CS_DISPATCH(g.Py, launch_fwd_y<PP>(f->F02, f->F13, f->tw[1], g, 1, st)); }
  if (cs_ngf_status s = check_launch("fwd_y (fixed)")) return s;
  { Stage sp(f, 6, st); CS_DISPATCH(g.Pz, launch_prep_z<PP>(f->F13, f->UV, f->tw[0], g, st)); }
  if (cs_ngf_status s = check_launch("prep_z")) return s;
  int sumA = 0;
  CS_CUDA(cudaMemcpyAsync(&sumA, f->msum, sizeof(int), cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaStreamSynchronize(st));
  if (sumA != f->sumA) {                 // the captured threshold launch holds sum(M_A)
    if (f->gexec) cudaGraphExecDestroy(f->gexec);
    f->gexec = nullptr;
    for (auto& gs : f->graphs) cudaGraphExecDestroy(gs.exec);
    f->graphs.clear();
  }
  f->sumA = sumA;
  return CS_NGF_OK;
}

// switch the handle to FFT lengths pad (each <= alloc_pad): twiddles, fixed
// spectra at the new lengths, and a new graph on the next full launch group
cs_ngf_status set_pads(cs_ngf_fixed* f, const int pad[3], cudaStream_t st) {
  Geo& g = f->g;
  const int cur[3] = {g.Pz, g.Py, g.Px};
  if (cur[0] == pad[0] && cur[1] == pad[1] && cur[2] == pad[2]) return CS_NGF_OK;
  CS_CUDA(cudaStreamSynchronize(st));            // nothing may still read the old tables
  for (int a = 0; a < 3; ++a)
    if (cur[a] != pad[a])
      if (cs_ngf_status s = fill_twiddles(pad[a], f->tw[a])) return s;
  // the captured launches hold the lengths: keep this graph for a later
  // return to them, and take the one of the new lengths if there is one
  if (f->gexec) {
    cs_ngf_fixed::GraphSlot gs{{g.Pz, g.Py, g.Px}, {0, 0, 0, 0, 0}, f->gexec};
    std::copy(f->gexec_vars, f->gexec_vars + kPasses, gs.vars);
    f->graphs.push_back(gs);
  }
  f->gexec = nullptr;
  for (size_t i = 0; i < f->graphs.size(); ++i)
    if (std::equal(pad, pad + 3, f->graphs[i].pad)) {
      f->gexec = f->graphs[i].exec;
      std::copy(f->graphs[i].vars, f->graphs[i].vars + kPasses, f->gexec_vars);
      f->graphs.erase(f->graphs.begin() + (long)i);
      break;
    }
  g.Pz = pad[0];
  g.Py = pad[1];
  g.Px = pad[2];
  resolve_variants(f);
  return run_fixed(f, f->A_keep, f->MA_keep, st);
}

// FP16 form: per channel field, the power of two that keeps the field's
// magnitude bound at most 2^15 (half of FP16's range) after the x pass
// (scale0) and after the y pass (scale1).  Per voxel a packed field has
// modulus at most 1 ((xx, yy), (zz, xy); Eq. 3's (x, y), (z, 0)) or 1/2
// ((xz, yz)), as the NGF is a unit vector or shorter (Eq. 1); a transform
// along an axis of n voxels multiplies the bound by at most n.
void set_field_scales(Geo& g) {
  for (int j = 0; j < 4; ++j) g.scale0[j] = g.scale1[j] = 1.0f;
  if (g.store != kStoreF16) return;
  for (int j = 0; j < g.nch; ++j) {
    const double b = (g.nch == 3 && j == 2) ? 0.5 : 1.0;
    const double b0 = b * g.nx, b1 = b * g.nx * (double)g.ny;
    g.scale0[j] = (float)std::ldexp(1.0, -std::max(0, (int)std::ceil(std::log2(b0 / 32768.0))));
    g.scale1[j] = (float)std::ldexp(1.0, -std::max(0, (int)std::ceil(std::log2(b1 / 32768.0))));
  }
}

// the shortest supported length >= need, at most cap
int length_for(int need, int cap) {
  for (int v : kPads)
    if (v >= need) return std::min(v, cap);
  return cap;
}

cs_ngf_status ensure_rotation_buffers(cs_ngf_fixed* f, int R) {
  if (R <= f->allb_cap) return CS_NGF_OK;
  CS_CUDA(cudaDeviceSynchronize());              // the old buffers may still be read
  cudaFree(f->allb);
  cudaFreeHost(f->allb_h);
  cudaFree(f->perm_d);
  cudaFree(f->perm_score);
  cudaFree(f->perm_shift);
  f->allb = f->perm_d = f->allb_h = nullptr;
  f->perm_score = nullptr;
  f->perm_shift = nullptr;
  f->allb_cap = 0;
  const int cap = std::max(R, 64);
  CS_CUDA(dalloc(&f->allb, (size_t)cap * 6));
  CS_CUDA(cudaMallocHost((void**)&f->allb_h, sizeof(int) * 6 * (size_t)cap));
  CS_CUDA(dalloc(&f->perm_d, (size_t)cap));
  CS_CUDA(dalloc(&f->perm_score, (size_t)cap));
  CS_CUDA(dalloc(&f->perm_shift, (size_t)cap * 3));
  f->allb_cap = cap;
  return CS_NGF_OK;
}

// Section 3.2 shift bounds of each of the R uploaded rotations (the same
// counts and bound the launch groups compute, from the floating volume
// pack_floating prepared) into f->allb_h [R][6]; synchronises st
cs_ngf_status rotation_bounds(cs_ngf_fixed* f, int R, cudaStream_t st) {
  if (cs_ngf_status s = ensure_rotation_buffers(f, R)) return s;
  const Geo& g = f->g;
  const size_t nmarg = (size_t)g.nz + g.ny + g.nx;
  for (int r0 = 0; r0 < R; r0 += f->batch) {
    const int nb = std::min(f->batch, R - r0);
    CS_CUDA(cudaMemsetAsync(f->msum, 0, sizeof(int) * nb, st));
    CS_CUDA(cudaMemsetAsync(f->margB, 0, sizeof(int) * nmarg * nb, st));
    {
      Stage sp(f, 0, st);
      k_mask_counts<<<resample_grid(g, nb), 128, 0, st>>>(f->C8, f->rot_d + r0, g, f->msum, f->margB);
    }
    if (cs_ngf_status s = check_launch("mask counts")) return s;
    {
      Stage sp(f, 7, st);
      k_shift_bounds<<<dim3((unsigned)nb, 3u), 512, 0, st>>>(f->margA, f->margB, f->msum, f->sumA,
                                                             f->gamma, g, f->allb + 6 * (size_t)r0);
    }
    if (cs_ngf_status s = check_launch("shift bounds")) return s;
  }
  CS_CUDA(cudaMemcpyAsync(f->allb_h, f->allb, sizeof(int) * 6 * (size_t)R, cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaStreamSynchronize(st));
  return CS_NGF_OK;
}

// FFT lengths one rotation needs: per axis the shortest supported P >=
// n + max(-chi_lo, chi_hi) over its admitted shifts; false if it admits none
bool rotation_lengths(const int dims[3], const int max_pad[3], const int* b, int pad[3]) {
  if (b[0] > b[1] || b[2] > b[3] || b[4] > b[5]) return false;
  for (int a = 0; a < 3; ++a) {
    const int n = dims[a], lo = b[2 * a], hi = b[2 * a + 1];
    pad[a] = length_for(n + std::max(n - 1 - lo, hi - (n - 1)), max_pad[a]);
  }
  return true;
}

cs_ngf_status check_volume_args(const cs_ngf_fixed* f, const float* B, const uint8_t* MB) {
  if (!f) return fail(CS_NGF_EINVAL, "handle is NULL");
  if (!B || !MB) return fail(CS_NGF_EINVAL, "B or maskB is NULL");
  return CS_NGF_OK;
}

// rotations [r0_begin, r0_begin + n) of the uploaded set; full launch groups
// replay the captured graph, a short tail is launched directly
cs_ngf_status score_range_impl(cs_ngf_fixed* f, int r0_begin, int n, float* best_score,
                               int32_t* best_shift, cudaStream_t st) {
  const int end = r0_begin + n;
  for (int r0 = r0_begin; r0 < end; r0 += f->batch) {
    const int nb = std::min(f->batch, end - r0);
    if (needs_tuning(f)) {                       // first group at these lengths: time the splits
      if (cs_ngf_status s = score_batch(f, r0, nb, best_score, best_shift, nullptr, st, true)) return s;
      continue;
    }
    if (nb == f->batch && !f->profiling) {
      if (cs_ngf_status s = ensure_graph(f)) return s;
      CS_CUDA(cudaMemcpyAsync(f->rot_slot, f->rot_d + r0, sizeof(RotMat) * nb, cudaMemcpyDeviceToDevice, st));
      CS_CUDA(cudaGraphLaunch(f->gexec, st));
      CS_CUDA(cudaMemcpyAsync(best_score + r0, f->slot_score, sizeof(float) * nb, cudaMemcpyDeviceToDevice, st));
      CS_CUDA(cudaMemcpyAsync(best_shift + 3 * (size_t)r0, f->slot_shift, sizeof(int32_t) * 3 * nb,
                              cudaMemcpyDeviceToDevice, st));
      g_launches.fetch_add(kKernelsPerBatch, std::memory_order_relaxed);
    } else if (cs_ngf_status s = score_batch(f, r0, nb, best_score, best_shift, nullptr, st)) {
      return s;
    }
  }
  return CS_NGF_OK;
}

// Bound-limited padding per rotation: each rotation's own shortest lengths;
// rotations that need the same lengths form one class, scored together.  A
// class costs a fixed-spectra recomputation, a stream synchronisation and
// (once per handle) a graph capture, about kClassCost rotations of its own
// size; so two classes merge, with lengths raised to cover both, while the
// cheapest merge adds less transform volume than that (and while there are
// more than kMaxClasses).  Rotations admitting no shift join the first
// class.  The classes do not depend on the launch-group size, so results
// stay the same for every even batch.
constexpr double kClassCost = 4.0;
constexpr size_t kMaxClasses = 8;
struct LengthClass { int pad[3]; std::vector<int> rot; };

double class_volume(const int* p) { return (double)p[0] * p[1] * p[2]; }

// dims, max_pad: the volume and the largest lengths; cur: the lengths in use
// (their class goes first); bounds [R][6]: each rotation's admitted shift
// slots {lo_z, hi_z, lo_y, hi_y, lo_x, hi_x}
std::vector<LengthClass> length_classes(const int dims[3], const int max_pad[3], const int cur[3],
                                        int R, const int* bounds) {
  std::vector<LengthClass> cls;
  std::vector<int> none;
  for (int r = 0; r < R; ++r) {
    int p[3];
    if (!rotation_lengths(dims, max_pad, bounds + 6 * (size_t)r, p)) { none.push_back(r); continue; }
    size_t k = 0;
    while (k < cls.size() && !std::equal(p, p + 3, cls[k].pad)) ++k;
    if (k == cls.size()) cls.push_back({{p[0], p[1], p[2]}, {}});
    cls[k].rot.push_back(r);
  }
  while (cls.size() > 1) {
    size_t bc = 0, bd = 1;
    double best = -1.0;
    int bm[3] = {0, 0, 0};
    for (size_t c = 0; c < cls.size(); ++c)
      for (size_t d = c + 1; d < cls.size(); ++d) {
        int m[3];
        for (int a = 0; a < 3; ++a) m[a] = std::max(cls[c].pad[a], cls[d].pad[a]);
        const double cost = (class_volume(m) - class_volume(cls[c].pad)) * cls[c].rot.size() +
                            (class_volume(m) - class_volume(cls[d].pad)) * cls[d].rot.size();
        if (best < 0.0 || cost < best) {
          best = cost;
          bc = c;
          bd = d;
          std::copy(m, m + 3, bm);
        }
      }
    const double keep = kClassCost * std::min(class_volume(cls[bc].pad), class_volume(cls[bd].pad));
    if (best >= keep && cls.size() <= kMaxClasses) break;
    std::copy(bm, bm + 3, cls[bc].pad);
    cls[bc].rot.insert(cls[bc].rot.end(), cls[bd].rot.begin(), cls[bd].rot.end());
    std::sort(cls[bc].rot.begin(), cls[bc].rot.end());
    cls.erase(cls.begin() + (long)bd);
  }
  if (cls.empty()) {
    LengthClass lc;
    for (int a = 0; a < 3; ++a) lc.pad[a] = length_for(dims[a], max_pad[a]);
    cls.push_back(lc);
  }
  cls[0].rot.insert(cls[0].rot.end(), none.begin(), none.end());
  std::sort(cls[0].rot.begin(), cls[0].rot.end());
  // start with the lengths in use (no recomputation), then the larger classes
  std::stable_sort(cls.begin(), cls.end(), [&](const LengthClass& a, const LengthClass& b) {
    const bool ca = std::equal(a.pad, a.pad + 3, cur), cb = std::equal(b.pad, b.pad + 3, cur);
    if (ca != cb) return ca;
    return a.rot.size() > b.rot.size();
  });
  return cls;
}

// Length classes of the R uploaded rotations (floating volume packed by
// pack_floating):
// bounds (synchronises st), classes, and the rotation matrices re-uploaded
// in class order when there is more than one.  perm[i] = original index of
// the i-th rotation in class order (empty if the order is unchanged); class
// c covers [ends[c-1], ends[c]) with lengths pads[c].  Without bound-limited
// padding: one class with the lengths in use.
cs_ngf_status plan_classes(cs_ngf_fixed* f, int R, cudaStream_t st,
                           std::vector<int>& perm, std::vector<int>& ends, std::vector<int>& pads) {
  perm.clear();
  ends.assign(1, R);
  pads.assign({f->g.Pz, f->g.Py, f->g.Px});
  f->length_sets = 1;
  f->last_pads = pads;
  f->last_counts.assign(1, R);
  if (f->pad_mode != CS_NGF_PAD_BOUND) return CS_NGF_OK;
  if (cs_ngf_status s = rotation_bounds(f, R, st)) return s;
  const int dims[3] = {f->g.nz, f->g.ny, f->g.nx}, cur[3] = {f->g.Pz, f->g.Py, f->g.Px};
  std::vector<LengthClass> cls = length_classes(dims, f->alloc_pad, cur, R, f->allb_h);
  f->length_sets = (int)cls.size();
  ends.clear();
  pads.clear();
  f->last_counts.clear();
  int k = 0;
  for (const auto& c : cls) {
    k += (int)c.rot.size();
    ends.push_back(k);
    pads.insert(pads.end(), c.pad, c.pad + 3);
    f->last_counts.push_back((int)c.rot.size());
  }
  f->last_pads = pads;
  if (cls.size() == 1) return CS_NGF_OK;
  // the stream is idle (rotation_bounds waited for it): rot_h is free
  std::vector<RotMat> orig(f->rot_h, f->rot_h + R);
  perm.reserve(R);
  k = 0;
  for (const auto& c : cls)
    for (int r : c.rot) { f->rot_h[k++] = orig[r]; perm.push_back(r); }
  CS_CUDA(cudaMemcpyAsync(f->rot_d, f->rot_h, sizeof(RotMat) * R, cudaMemcpyHostToDevice, st));
  CS_CUDA(cudaEventRecord(f->rot_ev, st));
  return CS_NGF_OK;
}

cs_ngf_status score_all(cs_ngf_fixed* f, const float* B, const uint8_t* MB, const double* quats,
                        int R, float* best_score, int32_t* best_shift, cudaStream_t st) {
  if (R <= 0) return fail(CS_NGF_EINVAL, "R must be positive");
  if (!best_score || !best_shift) return fail(CS_NGF_EINVAL, "output pointer is NULL");
  if (cs_ngf_status s = upload_rotations(f, quats, R, st)) return s;
  if (cs_ngf_status s = pack_floating(f, B, MB, st)) return s;
  std::vector<int> perm, ends, pads;
  if (cs_ngf_status s = plan_classes(f, R, st, perm, ends, pads)) return s;
  if (perm.empty()) {
    if (cs_ngf_status s = set_pads(f, pads.data(), st)) return s;
    return score_range_impl(f, 0, R, best_score, best_shift, st);
  }
  // classes one after another into the handle's buffers, then scattered to
  // the caller's order
  std::copy(perm.begin(), perm.end(), f->allb_h);   // pinned staging; the bounds are spent
  CS_CUDA(cudaMemcpyAsync(f->perm_d, f->allb_h, sizeof(int) * R, cudaMemcpyHostToDevice, st));
  int r0 = 0;
  for (size_t c = 0; c < ends.size(); ++c) {
    if (cs_ngf_status s = set_pads(f, pads.data() + 3 * c, st)) return s;
    if (cs_ngf_status s = score_range_impl(f, r0, ends[c] - r0, f->perm_score, f->perm_shift, st)) return s;
    r0 = ends[c];
  }
  { Stage sp(f, 7, st); k_scatter_results<<<(R + 255) / 256, 256, 0, st>>>(f->perm_d, f->perm_score, f->perm_shift, R, best_score, best_shift); }
  return check_launch("scatter results");
}

cs_ngf_status resolve_pads_impl(const int32_t dims[3], const cs_ngf_config& cfg, int pad[3]) {
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 2 || dims[a] > 256)
      return fail(CS_NGF_EINVAL, "dims must be in [2, 256], got " + std::to_string(dims[a]));
  if (!(cfg.eps > 0.0f) || !std::isfinite(cfg.eps)) return fail(CS_NGF_EINVAL, "eps must be > 0");
  if (!(cfg.gamma > 0.0f && cfg.gamma <= 1.0f)) return fail(CS_NGF_EINVAL, "gamma must be in (0, 1]");
  if (cfg.batch < 0) return fail(CS_NGF_EINVAL, "batch must be >= 0");
  if (cfg.measure != CS_NGF_SQUARED && cfg.measure != CS_NGF_UNSQUARED)
    return fail(CS_NGF_EINVAL, "unknown measure");
  if (cfg.precision != CS_NGF_FP32 && cfg.precision != CS_NGF_BF16 && cfg.precision != CS_NGF_FP16)
    return fail(CS_NGF_EINVAL, "unknown precision");
  if (cfg.pad_mode != CS_NGF_PAD_FULL && cfg.pad_mode != CS_NGF_PAD_BOUND)
    return fail(CS_NGF_EINVAL, "unknown pad_mode");
  if (cfg.autotune < 0 || cfg.autotune > 2) return fail(CS_NGF_EINVAL, "autotune must be 0, 1 or 2");
  if (cfg.tensor_cores != 0 && cfg.tensor_cores != 1) return fail(CS_NGF_EINVAL, "tensor_cores must be 0 or 1");
  for (int a = 0; a < 3; ++a) {
    pad[a] = cfg.pad[a] ? cfg.pad[a] : auto_pad(dims[a]);
    if (!pad_supported(pad[a]))
      return fail(CS_NGF_EUNSUPPORTED, "FFT length " + std::to_string(pad[a]) + " not supported");
    if (pad[a] < 2 * dims[a] - 1)
      return fail(CS_NGF_EINVAL, "FFT length " + std::to_string(pad[a]) + " < 2n-1");
  }
  return CS_NGF_OK;
}

struct Sizes {
  size_t f02_elems, f13_elems, fixed_f02, fixed_f13, per_rot, shared_ws, uv_elems;
  size_t zx_elems;   // X of the tensor-core z pass per rotation (0 when it is not used)
};

// channel fields per measure: three packed pairs of Eq. 6 products, or two of
// the Eq. 3 components; the mask field comes on top
int channel_fields(int measure) { return measure == CS_NGF_UNSQUARED ? 2 : 3; }

Sizes sizes_for(const int32_t dims[3], const int pad[3], int measure, int precision, int tensor_cores) {
  const size_t nz = dims[0], ny = dims[1], nx = dims[2];
  const size_t Pz = pad[0], Py = pad[1], Px = pad[2];
  const size_t vz = 2 * nz - 1, vy = 2 * ny - 1, nvox = nz * ny * nx;
  const size_t nch = channel_fields(measure), nf = nch + 1;
  const size_t cb = precision == CS_NGF_FP32 ? 8 : 4;            // bytes per channel value
  const size_t E0 = nz * ny * Px, E1 = nz * Px * Py;               // values per field of F0, F1
  Sizes z;
  z.f02_elems = (std::max((nch * cb + 8) * E0, vz * Px * Py * 8) + 7) / 8;
  z.f13_elems = (std::max((nch * cb + 8) * E1, vz * vy * Px * 8) + 7) / 8;
  z.fixed_f02 = nf * E0;                                            // one rotation, FP32 (A side)
  z.fixed_f13 = nf * E1;
  z.zx_elems = (tensor_cores && precision != CS_NGF_FP32) ? (Px / 2 + 1) * Py * Pz : 0;
  z.per_rot = (z.f02_elems + z.f13_elems + z.zx_elems) * sizeof(float2) + nvox * 5;
  z.shared_ws = nvox * (sizeof(float4) + 1);                       // BQ, C8
  z.uv_elems = (2 * nch + 1) * (Px / 2 + 1) * Py * Pz;
  return z;
}

cs_ngf_status ensure_results(cs_ngf_fixed* f, int R) {
  if (R <= f->res_cap) return CS_NGF_OK;
  CS_CUDA(cudaDeviceSynchronize());
  cudaFree(f->res_score);
  cudaFree(f->res_shift);
  f->res_score = nullptr;
  f->res_shift = nullptr;
  f->res_cap = 0;
  CS_CUDA(dalloc(&f->res_score, (size_t)R));
  CS_CUDA(dalloc(&f->res_shift, (size_t)R * 3));
  f->res_cap = R;
  return CS_NGF_OK;
}

}  // namespace

namespace csngf {
namespace detail {
cs_ngf_status upload_rotations(cs_ngf_fixed* f, const double* q, int R, cudaStream_t st) {
  return ::upload_rotations(f, q, R, st);
}
cs_ngf_status pack_floating(cs_ngf_fixed* f, const float* B, const uint8_t* MB, cudaStream_t st) {
  return ::pack_floating(f, B, MB, st);
}
cs_ngf_status score_range(cs_ngf_fixed* f, int r0, int n, float* best_score, int32_t* best_shift,
                          cudaStream_t st) {
  return ::score_range_impl(f, r0, n, best_score, best_shift, st);
}
cs_ngf_status plan_classes(cs_ngf_fixed* f, int R, cudaStream_t st,
                           std::vector<int>& perm, std::vector<int>& ends, std::vector<int>& pads) {
  return ::plan_classes(f, R, st, perm, ends, pads);
}
cs_ngf_status set_lengths(cs_ngf_fixed* f, const int pad[3], cudaStream_t st) {
  return ::set_pads(f, pad, st);
}
cs_ngf_status resolve_pads(const int32_t dims[3], const cs_ngf_config& cfg, int pad[3]) {
  return ::resolve_pads_impl(dims, cfg, pad);
}
size_t handle_bytes(const int32_t dims[3], const int pad[3], int batch, int measure, int precision,
                    int tensor_cores) {
  const Sizes z = ::sizes_for(dims, pad, measure, precision, tensor_cores);
  size_t tw = 0;
  for (int a = 0; a < 3; ++a) tw += (size_t)pad[a] * sizeof(float2);
  const size_t nmarg = (size_t)dims[0] + dims[1] + dims[2];
  const size_t keep = (size_t)dims[0] * dims[1] * dims[2] * 5;    // A, M_A copies (bound-limited padding)
  return z.uv_elems * sizeof(float2) + keep + (size_t)batch * z.per_rot + z.shared_ws +
         (size_t)batch * (sizeof(int) + sizeof(float) + sizeof(unsigned long long) + 6 * sizeof(int)) +
         (size_t)(batch + 1) * nmarg * sizeof(int) + tw;
}
}  // namespace detail
}  // namespace csngf

// ============================================================================
namespace {
// A call on a handle: claims it for this host thread (a second thread gets
// EBUSY and leaves the handle alone) and, with `order`, makes `st` wait for
// the event the previous call recorded on its own stream; on leaving, the
// call records that event on `st`.  Work of successive calls therefore never
// overlaps on the handle's buffers, whatever streams the calls use.
struct HandleCall {
  cs_ngf_fixed* f;
  cudaStream_t st;
  bool order;
  bool held = false;
  cudaError_t err = cudaSuccess;
  HandleCall(cs_ngf_fixed* h, cudaStream_t s, bool ord) : f(h), st(s), order(ord) {
    int idle = 0;
    held = f->busy.compare_exchange_strong(idle, 1, std::memory_order_acquire);
    if (held && order && f->order_ev) err = cudaStreamWaitEvent(st, f->order_ev, 0);
  }
  ~HandleCall() {
    if (!held) return;
    if (order && f->order_ev) cudaEventRecord(f->order_ev, st);
    f->busy.store(0, std::memory_order_release);
  }
};
}  // namespace

// claim handle f for this call (after its device is current); returns EBUSY
// or ECUDA from the calling function
#define CS_CLAIM(f, st, order)                                                         \
  HandleCall call_((f), (st), (order));                                                \
  if (!call_.held) return fail(CS_NGF_EBUSY, "another host thread is inside a call on this handle"); \
  if (call_.err != cudaSuccess)                                                        \
    return fail(CS_NGF_ECUDA, std::string("cudaStreamWaitEvent: ") + cudaGetErrorString(call_.err))

extern "C" {

static_assert(sizeof(cs_ngf_config) == 44, "cs_ngf_config layout (the Python binding mirrors it)");

void cs_ngf_default_config(cs_ngf_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->eps = 1e-5f;
  cfg->gamma = 0.5f;
  cfg->pad_mode = CS_NGF_PAD_BOUND;
  cfg->tensor_cores = 1;
}

int32_t cs_ngf_auto_pad(int32_t n) { return (n >= 2 && n <= 256) ? auto_pad(n) : 0; }

const char* cs_ngf_status_string(int32_t s) {
  switch (s) {
    case CS_NGF_OK: return "ok";
    case CS_NGF_EINVAL: return "invalid argument";
    case CS_NGF_ENOMEM: return "out of memory";
    case CS_NGF_ECUDA: return "CUDA error";
    case CS_NGF_ENOVALID: return "no valid shift for any rotation";
    case CS_NGF_EUNSUPPORTED: return "unsupported size";
    case CS_NGF_ECANCELED: return "cancelled";
    case CS_NGF_ETIMEOUT: return "timed out";
    case CS_NGF_EBUSY: return "handle busy";
    default: return "unknown status";
  }
}

const char* cs_ngf_last_error(void) { return g_last_error.c_str(); }

cs_ngf_status cs_ngf_prepare_fixed(const float* A, const uint8_t* maskA, const int32_t dims[3],
                                   const cs_ngf_config* cfg_in, void* stream, cs_ngf_fixed** out) {
  g_last_error.clear();
  if (!out) return fail(CS_NGF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A || !maskA || !dims) return fail(CS_NGF_EINVAL, "A, maskA or dims is NULL");
  cs_ngf_config cfg;
  cs_ngf_default_config(&cfg);
  if (cfg_in) cfg = *cfg_in;
  int pad[3];
  if (cs_ngf_status s = resolve_pads_impl(dims, cfg, pad)) return s;

  cs_ngf_fixed* f = new (std::nothrow) cs_ngf_fixed();
  if (!f) return fail(CS_NGF_ENOMEM, "host allocation failed");
  cudaGetDevice(&f->device);
  f->eps = cfg.eps;
  f->gamma = cfg.gamma;
  Geo& g = f->g;
  g.nz = dims[0]; g.ny = dims[1]; g.nx = dims[2];
  g.Pz = pad[0]; g.Py = pad[1]; g.Px = pad[2];
  g.vz = 2 * g.nz - 1; g.vy = 2 * g.ny - 1; g.vx = 2 * g.nx - 1;
  g.eps2 = cfg.eps * cfg.eps;
  g.nvox = (long long)g.nz * g.ny * g.nx;
  g.nch = channel_fields(cfg.measure);
  g.nf = g.nch + 1;
  g.store = cfg.precision == CS_NGF_BF16 ? kStoreBF16 : cfg.precision == CS_NGF_FP16 ? kStoreF16 : kStoreF32;
  set_field_scales(g);
  g.tc = cfg.tensor_cores;
  for (int a = 0; a < 3; ++a) f->alloc_pad[a] = pad[a];
  f->pad_mode = cfg.pad_mode;
  f->autotune = cfg.autotune;
  resolve_variants(f);

  const Sizes sz = sizes_for(dims, pad, cfg.measure, cfg.precision, cfg.tensor_cores);
  f->f02_elems = sz.f02_elems;
  f->f13_elems = sz.f13_elems;
  const size_t per_rot = sz.per_rot, shared_ws = sz.shared_ws, uv_elems = sz.uv_elems;
  int batch = cfg.batch;
  if (batch == 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t budget = free_b > uv_elems * sizeof(float2) ? (free_b - uv_elems * sizeof(float2)) / 3 : 0;
    batch = (int)std::max<size_t>(1, std::min<size_t>(32, budget / per_rot));
  }
  // launch grids index (rotation, field, z-plane) and (rotation, shift plane)
  // in their y dimension, at most 65535 blocks
  batch = std::min(batch, 65535 / std::max(g.nf * g.nz, 2 * g.nz - 1));
  // the masks of rotations 2k and 2k+1 share one transform; an even batch
  // keeps every pair inside one launch group, so results do not depend on it
  if (batch > 1 && (batch & 1)) --batch;
  f->batch = batch;

  cudaStream_t st = (cudaStream_t)stream;
  auto bail = [&](cs_ngf_status s) { std::string m = g_last_error; free_handle(f); g_last_error = m; return s; };
#define CS_TRY(call) do { cs_ngf_status s_ = (call); if (s_) return bail(s_); } while (0)
#define CS_TRYC(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return bail(fail( \
    e_ == cudaErrorMemoryAllocation ? CS_NGF_ENOMEM : CS_NGF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); } while (0)

  CS_TRYC(dalloc(&f->UV, uv_elems));
  CS_TRYC(dalloc(&f->Bh, (size_t)batch * g.nvox));
  CS_TRYC(dalloc(&f->Mh, (size_t)batch * g.nvox));
  CS_TRYC(dalloc(&f->BQ, (size_t)g.nvox));
  CS_TRYC(dalloc(&f->C8, (size_t)g.nvox));
  CS_TRYC(dalloc(&f->F02, std::max((size_t)batch * f->f02_elems, sz.fixed_f02)));
  CS_TRYC(dalloc(&f->F13, std::max((size_t)batch * f->f13_elems, sz.fixed_f13)));
  CS_TRYC(dalloc(&f->msum, (size_t)batch));
  const size_t nmarg = (size_t)g.nz + g.ny + g.nx;
  CS_TRYC(dalloc(&f->margA, nmarg));
  CS_TRYC(dalloc(&f->margB, (size_t)batch * nmarg));
  CS_TRYC(dalloc(&f->bounds, (size_t)batch * 6));
  CS_TRYC(dalloc(&f->thr, (size_t)batch));
  CS_TRYC(dalloc(&f->keys, (size_t)batch));
  if (sz.zx_elems) {
    CS_TRYC(dalloc(&f->zx, (size_t)batch * sz.zx_elems));
    g.zx = f->zx;
  }
  CS_TRYC(cudaEventCreateWithFlags(&f->order_ev, cudaEventDisableTiming));
  CS_TRYC(dalloc(&f->tc_err, (size_t)1));
  CS_TRYC(cudaMemsetAsync(f->tc_err, 0, sizeof(int), st));
  g.tc_err = f->tc_err;
  f->fixed_bytes = uv_elems * sizeof(float2);
  f->workspace_bytes = (size_t)batch * per_rot + shared_ws;
  for (int a = 0; a < 3; ++a) {                 // one table per axis: the lengths may part
    CS_TRYC(dalloc(&f->tw[a], (size_t)pad[a]));
    CS_TRY(fill_twiddles(pad[a], f->tw[a]));
  }
  if (f->pad_mode == CS_NGF_PAD_BOUND) {
    CS_TRYC(dalloc(&f->A_keep, (size_t)g.nvox));
    CS_TRYC(dalloc(&f->MA_keep, (size_t)g.nvox));
    CS_TRYC(cudaMemcpyAsync(f->A_keep, A, sizeof(float) * g.nvox, cudaMemcpyDeviceToDevice, st));
    CS_TRYC(cudaMemcpyAsync(f->MA_keep, maskA, (size_t)g.nvox, cudaMemcpyDeviceToDevice, st));
    f->fixed_bytes += (size_t)g.nvox * 5;
  }

  // A side into the new handle
  CS_TRY(run_fixed(f, A, maskA, st));
  CS_TRYC(cudaEventRecord(f->order_ev, st));
#undef CS_TRY
#undef CS_TRYC
  *out = f;
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_score_rotations(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                                     const double* quats, int32_t R, float* best_score,
                                     int32_t* best_shift, void* stream) {
  g_last_error.clear();
  if (cs_ngf_status s = check_volume_args(f, B, maskB)) return s;
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  return score_all(f, B, maskB, quats, R, best_score, best_shift, st);
}

cs_ngf_status cs_ngf_score_rotations_host(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                                          const double* quats, int32_t R, float* best_score,
                                          int32_t* best_shift, void* stream) {
  g_last_error.clear();
  if (cs_ngf_status s = check_volume_args(f, B, maskB)) return s;
  if (!best_score || !best_shift) return fail(CS_NGF_EINVAL, "output pointer is NULL");
  if (R <= 0) return fail(CS_NGF_EINVAL, "R must be positive");
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  if (!f->stage_B) {
    CS_CUDA(dalloc(&f->stage_B, (size_t)f->g.nvox));
    CS_CUDA(dalloc(&f->stage_M, (size_t)f->g.nvox));
  }
  if (cs_ngf_status s = ensure_results(f, R)) return s;
  CS_CUDA(cudaMemcpyAsync(f->stage_B, B, sizeof(float) * f->g.nvox, cudaMemcpyHostToDevice, st));
  CS_CUDA(cudaMemcpyAsync(f->stage_M, maskB, (size_t)f->g.nvox, cudaMemcpyHostToDevice, st));
  if (cs_ngf_status s = score_all(f, f->stage_B, f->stage_M, quats, R, f->res_score, f->res_shift, st))
    return s;
  CS_CUDA(cudaMemcpyAsync(best_score, f->res_score, sizeof(float) * R, cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaMemcpyAsync(best_shift, f->res_shift, sizeof(int32_t) * 3 * R, cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaStreamSynchronize(st));
  return tc_status(f, st);
}

cs_ngf_status cs_ngf_align(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                           const double* quats, int32_t R, float* score, int32_t* rot_index,
                           int32_t shift[3], void* stream) {
  g_last_error.clear();
  if (cs_ngf_status s = check_volume_args(f, B, maskB)) return s;
  if (!score || !rot_index || !shift) return fail(CS_NGF_EINVAL, "output pointer is NULL");
  if (R <= 0) return fail(CS_NGF_EINVAL, "R must be positive");
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  if (cs_ngf_status s = ensure_results(f, R)) return s;
  if (cs_ngf_status s = score_all(f, B, maskB, quats, R, f->res_score, f->res_shift, st)) return s;
  std::vector<float> sc(R);
  std::vector<int32_t> sh(3 * (size_t)R);
  CS_CUDA(cudaMemcpyAsync(sc.data(), f->res_score, sizeof(float) * R, cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaMemcpyAsync(sh.data(), f->res_shift, sizeof(int32_t) * 3 * R, cudaMemcpyDeviceToHost, st));
  CS_CUDA(cudaStreamSynchronize(st));
  if (cs_ngf_status s = tc_status(f, st)) return s;
  int best = -1;
  for (int r = 0; r < R; ++r)
    if (std::isfinite(sc[r]) && (best < 0 || sc[r] > sc[best])) best = r;
  if (best < 0) {
    *score = -INFINITY;
    *rot_index = -1;
    shift[0] = shift[1] = shift[2] = 0;
    return fail(CS_NGF_ENOVALID, "no rotation has a valid shift");
  }
  *score = sc[best];
  *rot_index = best;
  for (int a = 0; a < 3; ++a) shift[a] = sh[3 * (size_t)best + a];
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_score_map(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                               const double* quat, float* map, void* stream) {
  g_last_error.clear();
  if (cs_ngf_status s = check_volume_args(f, B, maskB)) return s;
  if (!map) return fail(CS_NGF_EINVAL, "map is NULL");
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  if (cs_ngf_status s = ensure_results(f, 1)) return s;
  if (cs_ngf_status s = upload_rotations(f, quat, 1, st)) return s;
  if (cs_ngf_status s = pack_floating(f, B, maskB, st)) return s;
  std::vector<int> perm, ends, pads;
  if (cs_ngf_status s = plan_classes(f, 1, st, perm, ends, pads)) return s;
  if (cs_ngf_status s = set_pads(f, pads.data(), st)) return s;
  return score_batch(f, 0, 1, f->res_score, f->res_shift, map, st);
}

cs_ngf_status cs_ngf_resample(cs_ngf_fixed* f, const float* B, const uint8_t* maskB,
                              const double* quat, float* Bhat, uint8_t* Mhat, void* stream) {
  g_last_error.clear();
  if (cs_ngf_status s = check_volume_args(f, B, maskB)) return s;
  if (!Bhat || !Mhat) return fail(CS_NGF_EINVAL, "output pointer is NULL");
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  if (cs_ngf_status s = upload_rotations(f, quat, 1, st)) return s;
  CS_CUDA(cudaMemsetAsync(f->msum, 0, sizeof(int), st));
  const Geo& g = f->g;
  if (cs_ngf_status s = pack_floating(f, B, maskB, st)) return s;
  k_resample<<<resample_grid(g, 1), 128, 0, st>>>(f->BQ, f->C8, f->rot_d, g, Bhat, Mhat, f->msum, nullptr);
  return check_launch("resample");
}

cs_ngf_status cs_ngf_get_info(const cs_ngf_fixed* f, cs_ngf_info* info) {
  if (!f || !info) return fail(CS_NGF_EINVAL, "handle or info is NULL");
  info->dims[0] = f->g.nz; info->dims[1] = f->g.ny; info->dims[2] = f->g.nx;
  info->pad[0] = f->g.Pz; info->pad[1] = f->g.Py; info->pad[2] = f->g.Px;
  info->batch = f->batch;
  info->sum_mask_a = f->sumA;
  info->fixed_bytes = (int64_t)f->fixed_bytes;
  info->workspace_bytes = (int64_t)f->workspace_bytes;
  for (int a = 0; a < 3; ++a) info->max_pad[a] = f->alloc_pad[a];
  info->pad_mode = f->pad_mode;
  info->length_sets = f->length_sets;
  info->reserved_ = 0;
  return CS_NGF_OK;
}

void cs_ngf_release(cs_ngf_fixed* f) { free_handle(f); }

int32_t cs_ngf_plan_lengths(const int32_t dims[3], const int32_t max_pad[3], const int32_t cur_pad[3],
                            int32_t R, const int32_t* bounds, int32_t cap, int32_t* pads,
                            int32_t* counts, int32_t* order) {
  if (!dims || !max_pad || R <= 0 || !bounds) return -1;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 2 || dims[a] > 256 || !pad_supported(max_pad[a]) || max_pad[a] < 2 * dims[a] - 1)
      return -1;
  const int d[3] = {dims[0], dims[1], dims[2]}, m[3] = {max_pad[0], max_pad[1], max_pad[2]};
  const int c[3] = {cur_pad ? cur_pad[0] : 0, cur_pad ? cur_pad[1] : 0, cur_pad ? cur_pad[2] : 0};
  const std::vector<LengthClass> cls = length_classes(d, m, c, R, bounds);
  int k = 0;
  for (size_t i = 0; i < cls.size(); ++i) {
    if ((int)i < cap) {
      if (pads)
        for (int a = 0; a < 3; ++a) pads[3 * i + a] = cls[i].pad[a];
      if (counts) counts[i] = (int32_t)cls[i].rot.size();
    }
    if (order)
      for (int r : cls[i].rot) order[k++] = r;
  }
  return (int32_t)cls.size();
}

int32_t cs_ngf_tuning(int32_t cap, cs_ngf_tuning_entry* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int n = 0;
  for (const auto& kv : g_tune) {
    if (out && n < cap) {
      cs_ngf_tuning_entry& e = out[n];
      e.pass = kv.first.pass;
      e.length = kv.first.P;
      e.half_input = kv.first.half;
      e.storage = kv.first.store;           // kStore* values equal the cs_ngf_precision codes
      e.variant = kv.second.variant;
      for (int v = 0; v < 2; ++v) {
        e.ms[v] = kv.second.ms[v];
        split_of(kv.first.P, v, &e.split[v][0], &e.split[v][1]);
      }
    }
    ++n;
  }
  return n;
}

void cs_ngf_tuning_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

int32_t cs_ngf_length_sets(const cs_ngf_fixed* f, int32_t cap, int32_t* pads, int32_t* counts) {
  if (!f) return 0;
  const int n = (int)f->last_counts.size();
  for (int c = 0; c < n && c < cap; ++c) {
    if (pads)
      for (int a = 0; a < 3; ++a) pads[3 * c + a] = f->last_pads[3 * (size_t)c + a];
    if (counts) counts[c] = f->last_counts[c];
  }
  return n;
}

cs_ngf_status cs_ngf_update_fixed(cs_ngf_fixed* f, const float* A, const uint8_t* maskA, void* stream) {
  g_last_error.clear();
  if (!f) return fail(CS_NGF_EINVAL, "handle is NULL");
  if (!A || !maskA) return fail(CS_NGF_EINVAL, "A or maskA is NULL");
  DeviceGuard guard(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  CS_CLAIM(f, st, true);
  if (f->A_keep) {                               // kept for later changes of FFT length
    CS_CUDA(cudaMemcpyAsync(f->A_keep, A, sizeof(float) * f->g.nvox, cudaMemcpyDeviceToDevice, st));
    CS_CUDA(cudaMemcpyAsync(f->MA_keep, maskA, (size_t)f->g.nvox, cudaMemcpyDeviceToDevice, st));
  }
  return run_fixed(f, A, maskA, st);
}

cs_ngf_status cs_ngf_set_profiling(cs_ngf_fixed* f, int32_t on) {
  if (!f) return fail(CS_NGF_EINVAL, "handle is NULL");
  CS_CLAIM(f, nullptr, false);
  f->profiling = on != 0;
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_stage_times(cs_ngf_fixed* f, double* ms, int64_t* launches) {
  if (!f || !ms || !launches) return fail(CS_NGF_EINVAL, "NULL argument");
  DeviceGuard guard(f->device);
  CS_CLAIM(f, nullptr, false);
  for (int i = 0; i < CS_NGF_NSTAGES; ++i) { ms[i] = 0.0; launches[i] = 0; }
  cs_ngf_status st = CS_NGF_OK;
  for (auto& sp : f->spans) {
    float t = 0.0f;
    if (cudaEventSynchronize(sp.b) != cudaSuccess || cudaEventElapsedTime(&t, sp.a, sp.b) != cudaSuccess)
      st = fail(CS_NGF_ECUDA, "event timing failed");
    if (sp.stage >= 0 && sp.stage < CS_NGF_NSTAGES) { ms[sp.stage] += t; launches[sp.stage] += 1; }
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  f->spans.clear();
  return st;
}

int64_t cs_ngf_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
