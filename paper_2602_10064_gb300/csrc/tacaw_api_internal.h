// Host-side internals shared by the translation units of libtacaw.so: the context, its
// caches, stream-ordered scratch and the error helpers.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"

namespace tacaw {
struct Serving;

// NVTX range over a scope of host code (an entry point or a phase of a run).  The calls only
// enqueue work, so a range marks the host-side issue of its launches; profilers that filter by
// range (ncu --nvtx --nvtx-include "tacaw_run/") select the kernels launched inside it.  Without
// an attached tool the push and pop do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}

struct GeoCache {
  using Band = tacaw::Band;
  Band band{}, aperture{};
  int* colnb = nullptr;
  float2* px = nullptr;   // [Wp] propagator along x for compact columns
  float2* py = nullptr;   // [ny]
  float2* mtab = nullptr; // [npair][ny][Wp]
  double* phix = nullptr;
  double* phiy = nullptr;
  double* coef_slots = nullptr;
  int32_t* qsel = nullptr;  // in-band q indices, ascending
  int64_t nsel = 0;
  int2* disc = nullptr;     // [ny]: (first index in qsel, count) of each grid row's in-band points
  int npair = 0, nslot = 0;
  uint64_t ff_version = 0;
};

// Per-kernel CUDA-event timing (diagnostics; off unless tacaw_profile_begin was called).
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
  double bytes, flops;
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<std::string> select;  // classes timed with events; empty: every class
};

// Pinned staging for the small host tables a run uploads (species slots, probe phase tables):
// a copy from pageable memory first waits for the stream's earlier work, which would make the
// launching thread wait for the GPU; from this ring the copy is asynchronous.  A region is
// reused only after the event recorded behind its copy has completed.
struct PinnedRing {
  unsigned char* base = nullptr;
  size_t cap = 0, head = 0;
  struct Span {
    size_t off, end;
    cudaEvent_t done;
  };
  std::vector<Span> inflight;          // in allocation order
  std::vector<cudaEvent_t> free_events;
};

struct tacaw_ctx {
  Profiler prof;
  PinnedRing staging;
  int device = 0;
  uint64_t budget = 0;
  std::string err;
  std::recursive_mutex mu;
  float2* tw = nullptr;  // FFT twiddles: length-N table at tw + tw_offset(N)
  std::vector<int32_t> ffZ;
  std::vector<double> ffcoef;
  int8_t* d_zslot = nullptr;  // form-factor slot of each Z in [0, 256), -1 if Z is not loaded
  uint64_t ff_version = 0;
  std::map<std::vector<double>, std::unique_ptr<GeoCache>> geos;
  std::map<int64_t, float2*> time_tw;
  std::map<int64_t, std::pair<void*, void*>> dft_ops;  // tensor-core DFT operands (hi, lo) per F and kind
  int* d_status = nullptr;  // device status word: bits TACAW_STATUS_* (tacaw_internal.cuh)
  int64_t max_chunk_frames = 0;  // option: cap on frames per chunk (0 = automatic)
  int64_t max_slice_block = 0;   // option: cap on slices per block of a run (0 = automatic)
  int64_t min_wave_rows = 0;     // option: wave rows a slice launch should hold (0 = default)
  int64_t max_run_bytes = 0;     // option: scratch bound of one run (0 = automatic)
  int64_t max_probe_block = 0;   // option: cap on the probes propagated and transformed together
  int64_t max_coalesce = 16;     // option: serving requests of one geometry coalesced into a run
  int64_t serving_streams = 4;   // option: streams per request class of the serving loop (before the first submit)
  int64_t serving_small_work = (int64_t)1 << 33;  // option: requests of at most this work are "small"
  int64_t static_band = 1;  // option: later-slice row passes built for the standard band (1) or not (0)
  int64_t host_copy = 1;  // option: results into page-locked host memory by 1 SM stores, 0 the copy engine
  std::vector<void*> owned;
  tacaw::Serving* serving = nullptr;
};


namespace tacaw {

// Stream-ordered scratch that frees itself on the stream.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <class T>
  cudaError_t get(T** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, sizeof(T) * std::max<size_t>(n, 1), st);
    if (e == cudaSuccess) ptrs.push_back(v);
    *p = static_cast<T*>(v);
    return e;
  }
};


// Records a CUDA event pair around the launches in its scope when profiling is on.
struct ProfScope {
  tacaw_ctx* ctx;
  cudaStream_t st;
  ProfRec rec{};
  bool active = false;
  ProfScope(tacaw_ctx* c, const char* name, cudaStream_t s, double bytes, double flops);
  ~ProfScope();
};

// Where the time transform reads its input and writes its output.  Column j < nsel of the
// transform reads psi[p][n][in_qsel ? in_qsel[j] : j] (row stride in_nq) and, for a full S,
// writes S[p][m][out_qsel ? out_qsel[j] : j] (row stride out_nq).  The run path reads a compact
// exit stack (in_nq = nsel, no in_qsel) and scatters into the full grid (out_qsel = the in-band
// q list); tacaw_spectrum uses the caller's q_sel on both sides.
struct SpecIO {
  int64_t in_nq;
  const int32_t* in_qsel;
  int64_t nsel;
  int64_t out_nq;
  const int32_t* out_qsel;
};

// Host -> device copy of `bytes` from pageable src through the context's pinned ring
// (asynchronous on st: src may be reused as soon as this returns).  Larger than the ring:
// a plain copy from pageable memory.
// n floats from device memory to host memory, stream-ordered: by SM stores when the option
// "host_copy" is 1 and dst is page-locked and mapped, else by cudaMemcpyAsync.
cudaError_t copy_to_host(tacaw_ctx* ctx, float* dst, const float* src, size_t n, cudaStream_t st);
// rows x width floats (pitches in floats) to dst, which may be host or device memory: SM stores
// for device memory and for mapped page-locked memory under "host_copy" 1, else
// cudaMemcpy2DAsync.
cudaError_t copy_rows_out(tacaw_ctx* ctx, float* dst, size_t dp, const float* src, size_t sp, size_t width,
                          size_t rows, cudaStream_t st);
cudaError_t staged_copy(tacaw_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st);

int set_err(tacaw_ctx* c, int code, const char* fmt, ...);
int cuda_err(tacaw_ctx* c, cudaError_t e, const char* where);
int get_time_tw(tacaw_ctx* ctx, int64_t F, float2** out);
// tensor-core time transform (k_dft_tc.cu)
// S: the full S (TACAW_REDUCE_NONE, written at the SpecIO output positions only) or the
// spectrum image SI[P][F] (TACAW_REDUCE_DETECTOR: the sum over the nsel columns, fused into the
// tensor-core epilogue).
int spectrum_tc(tacaw_ctx* ctx, const float2* psi_k, int64_t P, int64_t F, const SpecIO& io, int32_t precision,
                int32_t reduce, float* S, Scratch& sc);
// The whole time transform (mean, residual, DFT, |.|^2, optional detector sum) on P probes.
int spectrum_impl(tacaw_ctx* ctx, const float2* psi_k, int64_t P, int64_t F, const SpecIO& io, int32_t precision,
                  int32_t reduce, float* S_out, Scratch& sc);
// whole-path pieces (api.cu)
int get_geo(tacaw_ctx* ctx, const tacaw_params& p, GeoCache** out);
int check_run(tacaw_ctx* ctx, const tacaw_params* params, const tacaw_probe& pr, const float* pos,
              const int32_t* Z, int64_t n_atoms, int64_t n_frames, int32_t precision, int32_t reduce,
              const float* S_out, bool buffers);
// R trajectories of F frames each stacked along the frame axis run as one (shared launches);
// the output is [P][R][F][ny][nx] or [P][R][F].
uint64_t run_footprint(tacaw_ctx* ctx, const tacaw_params& p, int P, int64_t F, int64_t A, int32_t precision,
                       int32_t reduce, GeoCache* g, int R = 1);
int run_impl(tacaw_ctx* ctx, const tacaw_params& p, const tacaw_probe& pr, const float* d_pos, const int32_t* Z,
             bool z_dev, int64_t A, int64_t F, int32_t precision, int32_t reduce, float* d_S, cudaStream_t st,
             int R = 1);
// serving loop (serving.cpp)
void serving_shutdown(tacaw_ctx* ctx);

}  // namespace tacaw
