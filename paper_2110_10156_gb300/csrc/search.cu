// Global rigid alignment driver (Section 3.2): hybrid search where rotations
// are explored by random sampling around starting points and the best shift of
// each rotation comes from the all-shift similarity, inside a multi-level
// Gaussian pyramid (smoothing sigma_k, downsampling d_k, maximum step u_k,
// a_k random rotations, p_k starting points per level).  Each level keeps the
// best rotations of the previous one as its starting points and also scores
// those starting points themselves.
//
// Rotation parameters are Euler angles: about x, then the resulting y, then
// the resulting z (degrees).  Random numbers come from SplitMix64 (Steele, Lea
// and Flood 2014; constants as published by Vigna) so that a reference
// implementation can replay the same candidates.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/cs_ngf.h"
#include "handle.h"

using csngf::detail::fail;

namespace {

// ---------------------------------------------------------------- kernels
// 1D Gaussian along one axis, indices clamped at the faces
__global__ void k_gauss_axis(const float* __restrict__ in, float* __restrict__ out, int nz, int ny,
                             int nx, int axis, const float* __restrict__ w, int radius) {
  const long long n = (long long)nz * ny * nx;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((long long)nx * ny));
    float acc = 0.0f;
    for (int k = -radius; k <= radius; ++k) {
      int zz = z, yy = y, xx = x;
      if (axis == 0) zz = min(max(z + k, 0), nz - 1);
      else if (axis == 1) yy = min(max(y + k, 0), ny - 1);
      else xx = min(max(x + k, 0), nx - 1);
      acc += w[k + radius] * in[((long long)zz * ny + yy) * nx + xx];
    }
    out[i] = acc;
  }
}

// every d-th voxel (after the Gaussian), and the mask sampled at the same voxels
__global__ void k_subsample(const float* __restrict__ in, const uint8_t* __restrict__ min_,
                            int ny, int nx, int d, int oz, int oy, int ox, float* __restrict__ out,
                            uint8_t* __restrict__ mout) {
  const long long n = (long long)oz * oy * ox;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % ox);
    const int y = (int)((i / ox) % oy);
    const int z = (int)(i / ((long long)ox * oy));
    const long long s = ((long long)(d * z) * ny + d * y) * nx + d * x;
    out[i] = in[s];
    mout[i] = min_[s] ? 1 : 0;
  }
}

// ---------------------------------------------------------------- host math
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
};

// intrinsic x, then y', then z'' rotation -> unit quaternion (w, x, y, z)
void euler_to_quat(const double e_deg[3], double q[4]) {
  const double k = M_PI / 360.0;   // half angle in radians per degree
  const double cx = std::cos(e_deg[0] * k), sx = std::sin(e_deg[0] * k);
  const double cy = std::cos(e_deg[1] * k), sy = std::sin(e_deg[1] * k);
  const double cz = std::cos(e_deg[2] * k), sz = std::sin(e_deg[2] * k);
  // qx * qy
  const double a0 = cx * cy, a1 = sx * cy, a2 = cx * sy, a3 = sx * sy;
  // (qx qy) * qz
  q[0] = a0 * cz - a3 * sz;
  q[1] = a1 * cz + a2 * sz;
  q[2] = a2 * cz - a1 * sz;
  q[3] = a0 * sz + a3 * cz;
}

std::vector<float> gauss_weights(float sigma, int* radius) {
  const int r = (int)(4.0f * sigma + 0.5f);
  std::vector<float> w(2 * r + 1);
  double sum = 0.0;
  for (int k = -r; k <= r; ++k) sum += std::exp(-0.5 * (double)k * k / ((double)sigma * sigma));
  for (int k = -r; k <= r; ++k)
    w[k + r] = (float)(std::exp(-0.5 * (double)k * k / ((double)sigma * sigma)) / sum);
  *radius = r;
  return w;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
  template <class T> T* as() { return static_cast<T*>(p); }
};

#define SR_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? CS_NGF_ENOMEM : CS_NGF_ECUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// smooth (sigma > 0) then subsample by d; out buffers sized for the level
cs_ngf_status build_level(const float* V, const uint8_t* M, const int32_t dims[3], float sigma,
                          int d, float* tmp0, float* tmp1, float* out, uint8_t* mout,
                          const int32_t odims[3], cudaStream_t st) {
  const long long n = (long long)dims[0] * dims[1] * dims[2];
  const float* src = V;
  if (sigma > 0.0f) {
    int r = 0;
    std::vector<float> w = gauss_weights(sigma, &r);
    DevBuf dw;
    SR_CUDA(cudaMalloc(&dw.p, sizeof(float) * w.size()));
    SR_CUDA(cudaMemcpyAsync(dw.p, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, st));
    const float* in = V;
    float* bufs[2] = {tmp0, tmp1};
    for (int axis = 0; axis < 3; ++axis) {
      float* o = bufs[axis & 1];
      k_gauss_axis<<<1024, 256, 0, st>>>(in, o, dims[0], dims[1], dims[2], axis, dw.as<float>(), r);
      in = o;
    }
    SR_CUDA(cudaGetLastError());
    src = in;
    SR_CUDA(cudaStreamSynchronize(st));      // weights buffer is freed on return
  }
  (void)n;
  k_subsample<<<1024, 256, 0, st>>>(src, M, dims[1], dims[2], d, odims[0], odims[1], odims[2], out, mout);
  SR_CUDA(cudaGetLastError());
  return CS_NGF_OK;
}

}  // namespace

extern "C" {

void cs_ngf_search_default_config(cs_ngf_search_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  // the paper's schedule (Section 3.2 and 5.1 for NGF)
  c->levels = 4;
  const float sigma[4] = {5.0f, 3.0f, 2.0f, 1.5f};
  const int32_t d[4] = {4, 2, 2, 1};
  const float u[4] = {180.0f, 30.0f, 10.0f, 0.0f};
  const int32_t a[4] = {5000, 3000, 300, 0};
  const int32_t p[4] = {1, 20, 3, 1};
  for (int k = 0; k < 4; ++k) {
    c->sigma[k] = sigma[k];
    c->downsample[k] = d[k];
    c->max_step_deg[k] = u[k];
    c->random_rotations[k] = a[k];
    c->starting_points[k] = p[k];
  }
  c->seed = 0x5EEDull;
}

cs_ngf_status cs_ngf_global_align(const float* A, const uint8_t* maskA, const float* B,
                                  const uint8_t* maskB, const int32_t dims[3],
                                  const cs_ngf_config* cfg_in, const cs_ngf_search_config* scfg_in,
                                  void* stream, cs_ngf_search_result* out) {
  if (!A || !maskA || !B || !maskB || !dims || !out) return fail(CS_NGF_EINVAL, "NULL argument");
  cs_ngf_search_config sc;
  cs_ngf_search_default_config(&sc);
  if (scfg_in) sc = *scfg_in;
  if (sc.levels < 1 || sc.levels > CS_NGF_MAX_LEVELS) return fail(CS_NGF_EINVAL, "levels out of range");
  for (int k = 0; k < sc.levels; ++k) {
    if (sc.downsample[k] < 1 || sc.random_rotations[k] < 0 || sc.starting_points[k] < 1 ||
        sc.sigma[k] < 0.0f || sc.max_step_deg[k] < 0.0f)
      return fail(CS_NGF_EINVAL, "bad schedule at level " + std::to_string(k));
    for (int a = 0; a < 3; ++a)
      if ((dims[a] + sc.downsample[k] - 1) / sc.downsample[k] < 2)
        return fail(CS_NGF_EINVAL, "level " + std::to_string(k) + " is smaller than 2 voxels");
  }
  cs_ngf_config cfg;
  cs_ngf_default_config(&cfg);
  if (cfg_in) cfg = *cfg_in;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)dims[0] * dims[1] * dims[2];

  DevBuf t0, t1, la, lb, lma, lmb, rsc, rsh;
  SR_CUDA(cudaMalloc(&t0.p, sizeof(float) * n));
  SR_CUDA(cudaMalloc(&t1.p, sizeof(float) * n));
  SR_CUDA(cudaMalloc(&la.p, sizeof(float) * n));
  SR_CUDA(cudaMalloc(&lb.p, sizeof(float) * n));
  SR_CUDA(cudaMalloc(&lma.p, n));
  SR_CUDA(cudaMalloc(&lmb.p, n));

  SplitMix64 rng{sc.seed};
  std::vector<std::array<double, 3>> starts(1);
  for (int a = 0; a < 3; ++a) starts[0][a] = sc.start_euler_deg[a];
  std::memset(out, 0, sizeof(*out));
  out->score = -INFINITY;
  int64_t scored = 0;

  for (int k = 0; k < sc.levels; ++k) {
    const int d = sc.downsample[k];
    int32_t ld[3];
    for (int a = 0; a < 3; ++a) ld[a] = (dims[a] + d - 1) / d;
    if (cs_ngf_status s = build_level(A, maskA, dims, sc.sigma[k], d, t0.as<float>(), t1.as<float>(),
                                      la.as<float>(), lma.as<uint8_t>(), ld, st)) return s;
    if (cs_ngf_status s = build_level(B, maskB, dims, sc.sigma[k], d, t0.as<float>(), t1.as<float>(),
                                      lb.as<float>(), lmb.as<uint8_t>(), ld, st)) return s;
    // candidates: the starting points themselves, then a_k random steps around them
    std::vector<std::array<double, 3>> cand(starts);
    const double u = sc.max_step_deg[k];
    for (int i = 0; i < sc.random_rotations[k]; ++i) {
      const size_t pick = std::min(starts.size() - 1, (size_t)(rng.uniform() * (double)starts.size()));
      std::array<double, 3> e = starts[pick];
      for (int a = 0; a < 3; ++a) e[a] += (2.0 * rng.uniform() - 1.0) * u;
      cand.push_back(e);
    }
    const int R = (int)cand.size();
    std::vector<double> quats(4 * (size_t)R);
    for (int i = 0; i < R; ++i) euler_to_quat(cand[i].data(), &quats[4 * (size_t)i]);
    cs_ngf_config lc = cfg;
    lc.pad[0] = lc.pad[1] = lc.pad[2] = 0;   // each level takes its own automatic FFT lengths
    cs_ngf_fixed* h = nullptr;
    if (cs_ngf_status s = cs_ngf_prepare_fixed(la.as<float>(), lma.as<uint8_t>(), ld, &lc, st, &h)) return s;
    cudaFree(rsc.p);
    cudaFree(rsh.p);
    rsc.p = rsh.p = nullptr;
    cudaError_t e1 = cudaMalloc(&rsc.p, sizeof(float) * R);
    cudaError_t e2 = cudaMalloc(&rsh.p, sizeof(int32_t) * 3 * R);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cs_ngf_release(h);
      return fail(CS_NGF_ENOMEM, "result buffers");
    }
    cs_ngf_status s = cs_ngf_score_rotations(h, lb.as<float>(), lmb.as<uint8_t>(), quats.data(), R,
                                             rsc.as<float>(), rsh.as<int32_t>(), st);
    std::vector<float> hs(R);
    std::vector<int32_t> hh(3 * (size_t)R);
    if (!s) {
      cudaError_t e = cudaMemcpyAsync(hs.data(), rsc.p, sizeof(float) * R, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hh.data(), rsh.p, sizeof(int32_t) * 3 * R, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = fail(CS_NGF_ECUDA, cudaGetErrorString(e));
    }
    cs_ngf_release(h);
    if (s) return s;
    scored += R;
    // best first; equal scores keep the candidate order
    std::vector<int> order(R);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const bool fa = std::isfinite(hs[a]), fb = std::isfinite(hs[b]);
      if (fa != fb) return fa;
      return fa && hs[a] > hs[b];
    });
    const int keep = (k + 1 < sc.levels) ? sc.starting_points[k + 1] : 1;
    std::vector<std::array<double, 3>> next;
    for (int i = 0; i < R && (int)next.size() < keep; ++i) next.push_back(cand[order[i]]);
    starts.swap(next);
    const int b = order[0];
    out->level_best[k] = hs[b];
    if (k + 1 == sc.levels) {
      out->score = hs[b];
      for (int a = 0; a < 3; ++a) {
        out->euler_deg[a] = cand[b][a];
        out->shift[a] = hh[3 * (size_t)b + a] * d;
      }
      std::memcpy(out->quat, &quats[4 * (size_t)b], sizeof(out->quat));
    }
  }
  out->rotations_scored = scored;
  if (!std::isfinite(out->score)) return fail(CS_NGF_ENOVALID, "no valid shift at the last level");
  return CS_NGF_OK;
}

}  // extern "C"
