// Pipelined host-buffer stepping (locc_stepper_*): up to `depth` simulator
// steps in flight between page-locked host arrays and the device.  Each step
// takes one of `depth` slots of device staging (inputs, pair list, count,
// outputs):
//   copy-in stream:  wait until the slot's previous step has finished reading
//                    its inputs, copy poses / shapes / environment offsets in;
//   compute stream:  wait for the copy-in and for the slot's previous
//                    copy-out, run locc_step (broadphase, crop, network);
//   copy-out stream: wait for the step, copy the count, the pair list and the
//                    outputs out at the slot's full capacity (the count is only
//                    known on the device; the copy engine has the bandwidth).
// The steps themselves run one after another on the compute stream, since
// they share the handle's scratch; the copies of neighbouring steps overlap
// them.
#include <cstring>
#include <new>

#include "handle.cuh"

struct locc_stepper {
  locc_handle* h = nullptr;
  int depth = 0, max_pairs = 0, max_env = 0, max_obj = 0;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  struct Slot {
    char* dev = nullptr;  // poses | shapes | env offsets | count | pairs | out
    cudaEvent_t in_done = nullptr, run_done = nullptr, out_done = nullptr;
    int32_t* h_count = nullptr;  // page-locked
    int32_t* n_pairs_out = nullptr;
    long long ticket = -1;  // submitted and not yet waited for, else -1
    bool used = false;
  } slot[LOCC_STEPPER_MAX_DEPTH];
  size_t o_shape = 0, o_env = 0, o_cnt = 0, o_pairs = 0, o_out = 0, bytes = 0;
  long long next_ticket = 0;
};

namespace {

int sfail(int code, const char* msg) {
  locc::set_error(msg);
  return code;
}

#define STEP_TRY(expr)                                             \
  do {                                                             \
    if ((expr) != cudaSuccess) {                                   \
      cudaGetLastError();                                          \
      return sfail(LOCC_ERR_CUDA, "stepper: " #expr " failed");    \
    }                                                              \
  } while (0)

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

bool pinned(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

void stepper_free(locc_stepper* t) {
  for (int i = 0; i < LOCC_STEPPER_MAX_DEPTH; ++i) {
    auto& s = t->slot[i];
    if (s.dev) cudaFree(s.dev);
    if (s.h_count) cudaFreeHost(s.h_count);
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.run_done) cudaEventDestroy(s.run_done);
    if (s.out_done) cudaEventDestroy(s.out_done);
  }
  if (t->s_in) cudaStreamDestroy(t->s_in);
  if (t->s_run) cudaStreamDestroy(t->s_run);
  if (t->s_out) cudaStreamDestroy(t->s_out);
}

}  // namespace

extern "C" {

int locc_stepper_create(locc_handle* h, int32_t max_pairs, int32_t max_env, int32_t max_obj,
                        int32_t depth, locc_stepper** out) {
  if (!out) return sfail(LOCC_ERR_INVALID_ARG, "stepper: out is NULL");
  *out = nullptr;
  if (!h || max_pairs < 1 || max_env < 1 || max_obj < 1 || depth < 1 ||
      depth > LOCC_STEPPER_MAX_DEPTH)
    return sfail(LOCC_ERR_INVALID_ARG, "stepper: bad handle, size or depth");
  int st = locc_reserve(h, max_pairs, max_env);
  if (st) return st;
  locc_stepper* t = new (std::nothrow) locc_stepper();
  if (!t) return sfail(LOCC_ERR_OOM, "stepper: host allocation failed");
  t->h = h, t->depth = depth, t->max_pairs = max_pairs, t->max_env = max_env, t->max_obj = max_obj;
  t->o_shape = al256((size_t)max_obj * 28);
  t->o_env = t->o_shape + al256((size_t)max_obj * 4);
  t->o_cnt = t->o_env + al256((size_t)(max_env + 1) * 4);
  t->o_pairs = t->o_cnt + 256;
  t->o_out = t->o_pairs + al256((size_t)max_pairs * 8);
  t->bytes = t->o_out + al256((size_t)max_pairs * 32);
  bool ok = cudaStreamCreateWithFlags(&t->s_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&t->s_run, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&t->s_out, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < depth && ok; ++i) {
    auto& s = t->slot[i];
    ok = cudaMalloc(&s.dev, t->bytes) == cudaSuccess &&
         cudaMallocHost(&s.h_count, sizeof(int32_t)) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.run_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    stepper_free(t);
    delete t;
    return sfail(LOCC_ERR_OOM, "stepper: cannot allocate the slots");
  }
  *out = t;
  return LOCC_OK;
}

int locc_stepper_submit(locc_stepper* t, const float* poses, const int32_t* obj_shape,
                        int32_t n_obj, const int32_t* env_offsets, int32_t n_env,
                        int32_t* pairs_out, int32_t* n_pairs_out, float* out, int64_t* ticket) {
  if (!t || !ticket) return sfail(LOCC_ERR_INVALID_ARG, "stepper: stepper or ticket is NULL");
  if (n_obj < 0 || n_obj > t->max_obj || n_env < 0 || n_env > t->max_env)
    return sfail(LOCC_ERR_INVALID_ARG, "stepper: n_obj or n_env beyond the stepper's capacity");
  if (!n_pairs_out || !pinned(pairs_out) || !pinned(out) ||
      (n_obj > 0 && (!pinned(poses) || !pinned(obj_shape))) || !pinned(env_offsets))
    return sfail(LOCC_ERR_INVALID_ARG, "stepper: arrays must be page-locked host memory");
  int k = -1;  // a slot whose step has been waited for (any order of waits)
  for (int i = 0; i < t->depth && k < 0; ++i)
    if (t->slot[(t->next_ticket + i) % t->depth].ticket < 0) k = (int)((t->next_ticket + i) % t->depth);
  if (k < 0) return sfail(LOCC_ERR_BUSY, "stepper: all slots in flight; wait for one first");
  auto& s = t->slot[k];
  char* d = s.dev;
  if (s.used) STEP_TRY(cudaStreamWaitEvent(t->s_in, s.run_done, 0));  // inputs free again
  if (n_obj > 0) {
    STEP_TRY(cudaMemcpyAsync(d, poses, (size_t)n_obj * 28, cudaMemcpyHostToDevice, t->s_in));
    STEP_TRY(cudaMemcpyAsync(d + t->o_shape, obj_shape, (size_t)n_obj * 4, cudaMemcpyHostToDevice,
                             t->s_in));
  }
  STEP_TRY(cudaMemcpyAsync(d + t->o_env, env_offsets, (size_t)(n_env + 1) * 4,
                           cudaMemcpyHostToDevice, t->s_in));
  STEP_TRY(cudaEventRecord(s.in_done, t->s_in));
  STEP_TRY(cudaStreamWaitEvent(t->s_run, s.in_done, 0));
  if (s.used) STEP_TRY(cudaStreamWaitEvent(t->s_run, s.out_done, 0));  // outputs copied out
  int32_t* d_pairs = reinterpret_cast<int32_t*>(d + t->o_pairs);
  int32_t* d_cnt = reinterpret_cast<int32_t*>(d + t->o_cnt);
  float* d_out = reinterpret_cast<float*>(d + t->o_out);
  const int st = locc_step(t->h, reinterpret_cast<const float*>(d),
                           reinterpret_cast<const int32_t*>(d + t->o_shape), n_obj,
                           reinterpret_cast<const int32_t*>(d + t->o_env), n_env, d_pairs, d_cnt,
                           t->max_pairs, d_out, t->s_run);
  if (st) return st;
  STEP_TRY(cudaEventRecord(s.run_done, t->s_run));
  STEP_TRY(cudaStreamWaitEvent(t->s_out, s.run_done, 0));
  STEP_TRY(cudaMemcpyAsync(s.h_count, d_cnt, 4, cudaMemcpyDeviceToHost, t->s_out));
  STEP_TRY(cudaMemcpyAsync(pairs_out, d_pairs, (size_t)t->max_pairs * 8, cudaMemcpyDeviceToHost,
                           t->s_out));
  STEP_TRY(cudaMemcpyAsync(out, d_out, (size_t)t->max_pairs * 32, cudaMemcpyDeviceToHost, t->s_out));
  STEP_TRY(cudaEventRecord(s.out_done, t->s_out));
  s.used = true;
  s.n_pairs_out = n_pairs_out;
  s.ticket = t->next_ticket++;
  *ticket = s.ticket;
  return LOCC_OK;
}

int locc_stepper_wait(locc_stepper* t, int64_t ticket) {
  if (!t) return sfail(LOCC_ERR_INVALID_ARG, "stepper is NULL");
  for (int i = 0; i < t->depth; ++i) {
    auto& s = t->slot[i];
    if (s.ticket != ticket || ticket < 0) continue;
    STEP_TRY(cudaEventSynchronize(s.out_done));
    *s.n_pairs_out = *s.h_count;
    s.ticket = -1;
    return LOCC_OK;
  }
  return sfail(LOCC_ERR_INVALID_ARG, "stepper: no step in flight with this ticket");
}

void locc_stepper_destroy(locc_stepper* t) {
  if (!t) return;
  if (t->s_in) cudaStreamSynchronize(t->s_in);
  if (t->s_run) cudaStreamSynchronize(t->s_run);
  if (t->s_out) cudaStreamSynchronize(t->s_out);
  stepper_free(t);
  delete t;
}

}  // extern "C"
