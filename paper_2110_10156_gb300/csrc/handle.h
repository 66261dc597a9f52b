// Internal view of the library's handle, shared by its translation units
// (the C ABI only exposes it as an opaque pointer).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/cs_ngf.h"
#include "kernels.cuh"

struct cs_ngf_fixed {
  using Geo = csngf::Geo;
  using RotMat = csngf::RotMat;
  int device = 0;
  Geo g{};
  float eps = 1e-5f, gamma = 0.5f;
  int batch = 1;
  int sumA = 0;
  // FFT lengths the buffers are sized for (the automatic or requested ones);
  // g.Pz/Py/Px are the lengths in use, which bound-limited padding
  // (pad_mode CS_NGF_PAD_BOUND) lowers per call
  int alloc_pad[3] = {0, 0, 0};
  int pad_mode = 0;
  float* A_keep = nullptr;     // copies of A and M_A: the fixed spectra are
  uint8_t* MA_keep = nullptr;  // recomputed when the lengths in use change
  // per-rotation shift bounds of a call and its rotations regrouped by FFT
  // lengths (bound-limited padding), grown on demand to the call's R
  int* allb = nullptr;         // device [R][6]
  int* allb_h = nullptr;       // pinned host copy
  int* perm_d = nullptr;       // device: original index of each regrouped rotation
  float* perm_score = nullptr; // device results in regrouped order
  int32_t* perm_shift = nullptr;
  int allb_cap = 0;
  int length_sets = 1;         // sets of FFT lengths the last scoring call used
  std::vector<int> last_pads;  // their lengths [3 per set] and rotation counts
  std::vector<int> last_counts;
  // split variant of each FFT pass at the lengths in use (fwd_x, fwd_y, zmac,
  // inv_y, inv_x): 0 unless autotuning chose the alternative (autotune 1) or
  // the alternatives are requested outright (autotune 2)
  int autotune = 0;
  int vars[5] = {0, 0, 0, 0, 0};
  int gexec_vars[5] = {0, 0, 0, 0, 0};   // the variants gexec was captured with
  // one captured graph per set of FFT lengths (all reference the same buffers)
  struct GraphSlot { int pad[3]; int vars[5]; cudaGraphExec_t exec; };
  std::vector<GraphSlot> graphs;
  size_t f02_elems = 0, f13_elems = 0;
  float2* UV = nullptr;
  float* Bh = nullptr;
  uint8_t* Mh = nullptr;
  float4* BQ = nullptr;        // x-pairs of rows y, y+1 (B[i], B[i+1], B[i+sy], B[i+sy+1]) of the current call
  uint8_t* C8 = nullptr;       // corner codes of M_B of the current call
  float2* F02 = nullptr;
  float2* F13 = nullptr;
  int* msum = nullptr;
  int* margA = nullptr;        // slab counts of M_A per axis [nz | ny | nx]
  int* margB = nullptr;        // the same for each rotated mask of a batch
  int* bounds = nullptr;       // per rotation of a batch: shift slots that can be valid
  float* thr = nullptr;
  unsigned long long* keys = nullptr;
  int* tc_err = nullptr;       // set by a tensor-core pass that stopped on its bounded wait
  float2* zx = nullptr;        // X of the tensor-core z pass (reduced-precision forms), per launch group
  float2* tw[3] = {nullptr, nullptr, nullptr};   // z, y, x
  // rotation matrices: pinned host staging + device copy, grown on demand
  RotMat* rot_h = nullptr;
  RotMat* rot_d = nullptr;
  int rot_cap = 0;
  cudaEvent_t rot_ev = nullptr;
  // host-buffer entry point staging
  float* stage_B = nullptr;
  uint8_t* stage_M = nullptr;
  float* res_score = nullptr;
  int32_t* res_shift = nullptr;
  int res_cap = 0;
  size_t fixed_bytes = 0, workspace_bytes = 0;
  // one captured CUDA graph for a full batch, replayed per batch; the batch's
  // rotation matrices and results go through fixed slots
  cudaGraphExec_t gexec = nullptr;
  RotMat* rot_slot = nullptr;
  float* slot_score = nullptr;
  int32_t* slot_shift = nullptr;
  bool capturing = false;
  // per-stage CUDA-event timing (cs_ngf_set_profiling); disables graph replay
  bool profiling = false;
  struct Span { int stage; cudaEvent_t a, b; };
  std::vector<Span> spans;
  // one call at a time: set while a host thread is inside a call on this
  // handle (a second thread gets CS_NGF_EBUSY)
  std::atomic<int> busy{0};
  // recorded on the caller's stream at the end of every call; the next call
  // waits for it on its own stream, so calls on different streams do not
  // overlap on the workspace
  cudaEvent_t order_ev = nullptr;
};

namespace csngf {
namespace detail {

// record the calling thread's error detail (cs_ngf_last_error) and return s
cs_ngf_status fail(cs_ngf_status s, const std::string& msg);
// host FP64 quaternions -> FP32 matrices in f->rot_d[0..R)
cs_ngf_status upload_rotations(cs_ngf_fixed* f, const double* quats, int R, cudaStream_t st);
// (B, M_B) -> f->BQ, f->C8 for the following score calls
cs_ngf_status pack_floating(cs_ngf_fixed* f, const float* B, const uint8_t* MB, cudaStream_t st);
// Bound-limited padding (pad_mode CS_NGF_PAD_BOUND): the R uploaded
// rotations of the floating volume packed by pack_floating, grouped into
// classes by the FFT lengths their admitted shifts need.  Synchronises `st`.  perm[i] is the
// original index of the i-th rotation in class order (empty: order
// unchanged; otherwise the device matrices are re-uploaded in that order);
// class c covers [ends[c-1], ends[c]) and uses lengths pads[3c..3c+2].  In
// other modes: one class with the lengths in use.
cs_ngf_status plan_classes(cs_ngf_fixed* f, int R, cudaStream_t st,
                           std::vector<int>& perm, std::vector<int>& ends, std::vector<int>& pads);
// switch the handle to FFT lengths pad (recomputing the fixed spectra if they
// change; synchronises `st` then)
cs_ngf_status set_lengths(cs_ngf_fixed* f, const int pad[3], cudaStream_t st);
// score rotations [r0, r0 + n) of the uploaded set into best_score / best_shift
// (device, indexed from r0), in launch groups of f->batch
cs_ngf_status score_range(cs_ngf_fixed* f, int r0, int n, float* best_score, int32_t* best_shift,
                          cudaStream_t st);
// validate dims / cfg and return the FFT lengths; EINVAL / EUNSUPPORTED on error
cs_ngf_status resolve_pads(const int32_t dims[3], const cs_ngf_config& cfg, int pad[3]);
// device bytes a handle of these dims, FFT lengths and batch allocates
size_t handle_bytes(const int32_t dims[3], const int pad[3], int batch, int measure, int precision,
                    int tensor_cores);

}  // namespace detail
}  // namespace csngf
