// Epoch hand-over (Sec. "High-level Genetic Algorithm loop": iterations are
// grouped into epochs, and only at an epoch's end do results leave the GPU for
// the AC optimiser, so the device loop is not interrupted by a transfer after
// every iteration).
//
// tto_epoch_export queues, on the caller's stream and in order after the
// epoch's iterations, a device-to-device snapshot of the archive (fitness,
// genomes, filled flags) and the worst-k N-1 cases of every cell's genome
// (tto_worst_k).  It then copies the snapshot to host memory on a side stream
// that waits for it by event.  The next epoch's iterations, queued on the
// caller's stream, overlap the transfer.  A later export first makes the
// caller's stream wait for the previous transfer (device-side, by event) so
// the snapshot is never overwritten while it is being copied out.  There are
// no spin-waits: only events and stream ordering.
#include "tto_internal.h"

namespace tto {

struct EpochSnap {
  int k = 0;
  float* fit = nullptr;      // [cells]
  int32_t* gen = nullptr;    // [cells][gw]
  uint8_t* filled = nullptr; // [cells]
  int32_t* widx = nullptr;   // [cells][k]
  float* wval = nullptr;     // [cells][k]
  cudaStream_t side = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  bool pending = false;
};

void free_epoch(tto_archive* a) {
  EpochSnap* e = a->epoch;
  if (!e) return;
  if (e->pending && e->done) cudaEventSynchronize(e->done);
  void* ptrs[] = {e->fit, e->gen, e->filled, e->widx, e->wval};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (e->side) cudaStreamDestroy(e->side);
  if (e->ready) cudaEventDestroy(e->ready);
  if (e->done) cudaEventDestroy(e->done);
  delete e;
  a->epoch = nullptr;
}

}  // namespace tto

using namespace tto;


extern "C" int tto_epoch_export(tto_archive* a, int32_t k, float* fitness, int32_t* genome, uint8_t* filled,
                                int32_t* worst_outage, float* worst_energy, void* stream) {
  if (!a || k < 0 || k > 1024) return set_error(TTO_E_ARG, "bad epoch export arguments");
  if (!fitness || !genome || !filled || (k > 0 && (!worst_outage || !worst_energy)))
    return set_error(TTO_E_ARG, "null host buffer");
  tto_grid* g = a->g;
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  const size_t C = a->cells, gw = g->gw;
  if (!a->epoch) {
    a->epoch = new (std::nothrow) EpochSnap();
    if (!a->epoch) return set_error(TTO_E_NOMEM, "host allocation failed");
    EpochSnap* e = a->epoch;
    TTO_CUDA_TRY(cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking));
    TTO_CUDA_TRY(cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming));
    TTO_CUDA_TRY(cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming));
    TTO_CUDA_TRY(cudaMalloc(&e->fit, C * sizeof(float)));
    TTO_CUDA_TRY(cudaMalloc(&e->gen, C * gw * sizeof(int32_t)));
    TTO_CUDA_TRY(cudaMalloc(&e->filled, C));
  }
  EpochSnap* e = a->epoch;
  if (e->pending) TTO_CUDA_TRY(cudaStreamWaitEvent(s, e->done, 0));  // the previous copy-out has finished
  if (k > e->k) {
    if (e->pending) TTO_CUDA_TRY(cudaEventSynchronize(e->done));
    if (e->widx) cudaFree(e->widx);
    if (e->wval) cudaFree(e->wval);
    e->widx = nullptr;
    e->wval = nullptr;
    e->k = 0;
    TTO_CUDA_TRY(cudaMalloc(&e->widx, C * k * sizeof(int32_t)));
    TTO_CUDA_TRY(cudaMalloc(&e->wval, C * k * sizeof(float)));
    e->k = k;
  }
  TTO_CUDA_TRY(cudaMemcpyAsync(e->fit, a->d_fit, C * sizeof(float), cudaMemcpyDeviceToDevice, s));
  TTO_CUDA_TRY(cudaMemcpyAsync(e->gen, a->d_genome, C * gw * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  TTO_CUDA_TRY(cudaMemcpyAsync(e->filled, a->d_filled, C, cudaMemcpyDeviceToDevice, s));
  if (k > 0) {
    // empty cells are skipped: their lists come out as -1 / NaN
    const int rc = worst_k_impl(g, e->gen, (int32_t)C, nullptr, 0, k, e->widx, e->wval, nullptr, e->filled, s);
    if (rc) return rc;
  }
  TTO_CUDA_TRY(cudaEventRecord(e->ready, s));
  TTO_CUDA_TRY(cudaStreamWaitEvent(e->side, e->ready, 0));
  TTO_CUDA_TRY(cudaMemcpyAsync(fitness, e->fit, C * sizeof(float), cudaMemcpyDeviceToHost, e->side));
  TTO_CUDA_TRY(cudaMemcpyAsync(genome, e->gen, C * gw * sizeof(int32_t), cudaMemcpyDeviceToHost, e->side));
  TTO_CUDA_TRY(cudaMemcpyAsync(filled, e->filled, C, cudaMemcpyDeviceToHost, e->side));
  if (k > 0) {
    TTO_CUDA_TRY(cudaMemcpyAsync(worst_outage, e->widx, C * k * sizeof(int32_t), cudaMemcpyDeviceToHost, e->side));
    TTO_CUDA_TRY(cudaMemcpyAsync(worst_energy, e->wval, C * k * sizeof(float), cudaMemcpyDeviceToHost, e->side));
  }
  TTO_CUDA_TRY(cudaEventRecord(e->done, e->side));
  e->pending = true;
  return TTO_OK;
}

extern "C" int tto_epoch_export_wait(tto_archive* a) {
  if (!a) return set_error(TTO_E_ARG, "null archive");
  if (!a->epoch || !a->epoch->pending) return TTO_OK;
  TTO_CUDA_TRY(cudaSetDevice(a->g->device));
  TTO_CUDA_TRY(cudaEventSynchronize(a->epoch->done));
  a->epoch->pending = false;
  return TTO_OK;
}
