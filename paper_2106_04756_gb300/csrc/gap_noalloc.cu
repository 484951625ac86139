// pdlp_normalized_gap_noalloc: the normalized duality gap with no device
// allocation.  Its scratch lives in one file-scope __device__ array instead of
// memory obtained from cudaMalloc.
//
// Some callers cannot allocate device memory: a host application whose
// framework allocator already owns (or has reserved) all of the GPU's memory,
// or a latency-bound caller that cannot afford cudaMalloc / cudaFree and the
// device-wide synchronisation they may imply.  This call serves them: the
// caller passes device inputs and host outputs, and the library uses only the
// static array below.
//
// Scratch layout (g_gap_scratch, kScratchBytes, held by every GPU that loads
// the library until the process exits):
//   [0, 256)          selection state (GapState)
//   [256, 512)        arrival counter of the pass kernel
//   [512, +48 KiB)    histogram, 3 x 2048 float64
//   then              float32 keys of up to kNoallocMaxItems coordinates
#include <math.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace pdlp {
void set_last_error(const std::string &msg);  // api.cu: message for pdlp_last_error(NULL)
}

namespace {

constexpr int kNoallocMaxItems = 1 << 20;  // n + m limit of the call
constexpr int kNB = 2048;                  // digit buckets
constexpr int kPassThreads = 512;
constexpr size_t kStateOff = 0, kTicketOff = 256, kHistOff = 512;
constexpr size_t kKeysOff = kHistOff + sizeof(double) * 3 * kNB;
constexpr size_t kScratchBytes = kKeysOff + sizeof(unsigned) * (size_t)kNoallocMaxItems;
constexpr int kMaxDevices = 64;

struct GapState {
  double r2, omega, W, V, A, mu, value;
  unsigned prefix;
};

static __device__ __align__(256) unsigned char g_gap_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

struct Inputs {
  int32_t n, m;
  const double *x, *y, *gx, *gy, *l, *u, *ylo;
};

struct Item {
  unsigned key;  // float bits of the breakpoint t_i, 0xffffffff = no item
  double a, w, v;
};

// Coordinate i of the trust-region problem (Section 3.2): a (coefficient of t^2
// in phi and of t in the gap while unclipped), w, v (contributions once
// clipped) and the breakpoint key.  Same item set as the library's gap: a
// coordinate that cannot move, or whose float breakpoint is not positive,
// gives no item.
__device__ __forceinline__ Item make_item(const Inputs &in, double om, int i) {
  Item it;
  it.key = 0xffffffffu;
  it.a = it.w = it.v = 0.0;
  double g, dist;
  bool primal = i < in.n;
  if (primal) {
    g = in.gx[i];
    if (g == 0.0) return it;
    dist = g > 0.0 ? in.u[i] - in.x[i] : in.x[i] - in.l[i];
  } else {
    const int r = i - in.n;
    g = in.gy[r];
    if (g == 0.0) return it;
    dist = g > 0.0 ? INFINITY : in.y[r] - in.ylo[r];
  }
  // a coordinate on its bound in the ascent direction (or an ulp past it)
  // cannot move: no item, as in the library's gap
  if (!(dist > 0.0)) return it;
  const double ag = fabs(g);
  if (isinf(dist)) {
    it.a = primal ? g * g / om : om * g * g;
    it.key = 0x7f800000u;
    return it;
  }
  const float tf = primal ? (float)(om * dist) / (float)ag : (float)dist / ((float)om * (float)ag);
  if (!(tf > 0.0f)) return it;  // breakpoint below float resolution: no item, as in the library's gap
  it.a = primal ? g * g / om : om * g * g;
  it.key = __float_as_uint(tf);
  it.w = primal ? om * dist * dist : dist * dist / om;
  it.v = ag * dist;
  return it;
}

__global__ void k_nag_clear(unsigned char *scratch, double r2, double omega) {
  double *h = reinterpret_cast<double *>(scratch + kHistOff);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < 3 * kNB; b += gridDim.x * blockDim.x) h[b] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    GapState *s = reinterpret_cast<GapState *>(scratch + kStateOff);
    s->r2 = r2;
    s->omega = omega;
    s->W = s->V = s->A = 0.0;
    s->mu = s->value = 0.0;
    s->prefix = 0u;
    *reinterpret_cast<unsigned *>(scratch + kTicketOff) = 0u;
  }
}

// One radix pass over all coordinates (11, 11, 10 bits of the float key),
// shared-memory histogram flushed to the scratch histogram; the last CTA picks
// the last bucket whose lower edge has phi < r^2 and clears the histogram.
constexpr int kPassSmem = (int)(sizeof(double) * (4 * kNB + 8));

__global__ void __launch_bounds__(kPassThreads) k_nag_pass(Inputs in, unsigned char *scratch, int pass) {
  extern __shared__ __align__(16) double hs[];  // 3 x kNB histogram, then kNB + 1 suffix sums
  GapState *st = reinterpret_cast<GapState *>(scratch + kStateOff);
  unsigned *ticket = reinterpret_cast<unsigned *>(scratch + kTicketOff);
  double *gh = reinterpret_cast<double *>(scratch + kHistOff);
  unsigned *keys = reinterpret_cast<unsigned *>(scratch + kKeysOff);
  const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
  const int nb = pass == 2 ? 1024 : 2048;
  const int pshift = pass == 1 ? 21 : 10;
  const unsigned pref = pass == 0 ? 0u : st->prefix >> pshift;
  const double om = st->omega;
  for (int e = threadIdx.x; e < 3 * kNB; e += blockDim.x) hs[e] = 0.0;
  __syncthreads();
  const int N = in.n + in.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    Item it;
    if (pass == 0) {
      it = make_item(in, om, i);
      keys[i] = it.key;
      if (it.key == 0xffffffffu) continue;
    } else {
      const unsigned key = keys[i];
      if (key == 0xffffffffu || (key >> pshift) != pref) continue;
      it = make_item(in, om, i);
    }
    const int b = (int)((it.key >> shift) & (unsigned)(nb - 1));
    atomicAdd(hs + b, it.w);
    atomicAdd(hs + kNB + b, it.v);
    atomicAdd(hs + 2 * kNB + b, it.a);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const double v = hs[a * kNB + b];
      if (v != 0.0) atomicAdd(gh + (size_t)b * 3 + a, v);
    }
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(ticket, 1u);
    s_last = prev == gridDim.x - 1;
    if (s_last) *ticket = 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int b = threadIdx.x; b < kNB; b += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      hs[a * kNB + b] = b < nb ? __ldcg(gh + (size_t)b * 3 + a) : 0.0;
      gh[(size_t)b * 3 + a] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const unsigned base = pass == 0 ? 0u : (st->prefix >> (pass == 1 ? 21 : 10)) << (pass == 1 ? 21 : 10);
  double *suf = hs + 3 * kNB;  // suf[b] = A_above + sum of a over buckets >= b
  suf[nb] = st->A;
  for (int b = nb - 1; b >= 0; --b) suf[b] = suf[b + 1] + hs[2 * kNB + b];
  int best = 0;
  double Wb = st->W, Vb = st->V, Wbest = Wb, Vbest = Vb;
  for (int b = 0; b < nb; ++b) {
    const double Tb = (double)__uint_as_float(base | ((unsigned)b << shift));
    const double phi = suf[b] > 0.0 ? Wb + Tb * Tb * suf[b] : Wb;
    if (!(phi < st->r2)) break;
    best = b;
    Wbest = Wb;
    Vbest = Vb;
    Wb += hs[b];
    Vb += hs[kNB + b];
  }
  const double Aafter = suf[best + 1];
  st->W = Wbest;
  st->V = Vbest;
  st->A = Aafter;
  st->prefix = base | ((unsigned)best << shift);
  if (pass == 2) {
    const double Wf = Wbest + hs[best], Vf = Vbest + hs[kNB + best];
    double val = Vf;
    if (Aafter > 0.0) {
      const double rem = st->r2 - Wf;
      val = Vf + sqrt((rem > 0.0 ? rem : 0.0) / Aafter) * Aafter;
    }
    st->value = val;
    st->mu = val / sqrt(st->r2);
  }
}

int fail(int code, const std::string &msg) {
  pdlp::set_last_error(msg);
  return code;
}

// Set-up, once per device with that device current: the device address of the
// static scratch (a host-side name of a __device__ array is not a device
// address) and the pass kernel's shared-memory size.  Cached afterwards.
int scratch_for_current_device(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PDLP_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gap_scratch);
    if (e != cudaSuccess || !p)
      return fail(PDLP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaFuncSetAttribute(k_nag_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    if (e != cudaSuccess)
      return fail(PDLP_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PDLP_OK;
}

}  // namespace

extern "C" int pdlp_normalized_gap_noalloc(int32_t n, int32_t m, const double *x, const double *y,
                                           const double *gx, const double *gy, const double *l,
                                           const double *u, const double *ylo, double omega, double r,
                                           void *stream, double *mu, double *value) {
  if (n < 0 || m < 0 || !mu) return fail(PDLP_ERR_INVALID_ARG, "n, m must be >= 0 and mu non-NULL");
  if ((int64_t)n + (int64_t)m > kNoallocMaxItems)
    return fail(PDLP_ERR_INVALID_ARG, "pdlp_normalized_gap_noalloc: n + m = " + std::to_string((int64_t)n + m) +
                                          " exceeds the static scratch limit of " +
                                          std::to_string(kNoallocMaxItems) + " coordinates");
  if (!(r > 0.0) || !(omega > 0.0)) return fail(PDLP_ERR_INVALID_ARG, "r and omega must be > 0");
  if ((n > 0 && (!x || !gx || !l || !u)) || (m > 0 && (!y || !gy || !ylo)))
    return fail(PDLP_ERR_INVALID_ARG, "NULL input array");
  void *scr = nullptr;
  int rc = scratch_for_current_device(&scr);
  if (rc) return rc;
  unsigned char *s = reinterpret_cast<unsigned char *>(scr);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Inputs in{n, m, x, y, gx, gy, l, u, ylo};
  k_nag_clear<<<8, 256, 0, st>>>(s, r * r, omega);
  const int N = n + m;
  int grid = (N + kPassThreads - 1) / kPassThreads;
  if (grid > 304) grid = 304;
  if (grid < 1) grid = 1;
  for (int pass = 0; pass < 3; ++pass) k_nag_pass<<<grid, kPassThreads, kPassSmem, st>>>(in, s, pass);
  GapState hs;
  cudaError_t e = cudaMemcpyAsync(&hs, s + kStateOff, sizeof(GapState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? PDLP_ERR_OOM : PDLP_ERR_CUDA,
                std::string("pdlp_normalized_gap_noalloc: ") + cudaGetErrorString(e));
  *mu = hs.mu;
  if (value) *value = hs.value;
  return PDLP_OK;
}
