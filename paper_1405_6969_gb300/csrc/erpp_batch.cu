// erpp_batch.cu -- many independent boxes stepped together.
//
// A batch owns one context per box (its own scratch, sized at creation for
// the box's particle count) and the box descriptors.  erpp_step_batched runs
// the coupling step of every box.  With a graph, the first call for a given
// first_step value captures all boxes' launch sequences once into one CUDA
// graph: a fork node, one independent branch per box (bin, gather, removal
// + drag + advance, scatter, halo merge, each box on its own capture
// stream), and a join.  Later calls replay that graph with one launch on the
// caller's stream, so the host issues one launch per step whatever the
// number of boxes, and small boxes that cannot fill the GPU alone run
// concurrently.  Without a graph the same sequences are issued box after box
// on the caller's stream (plain launches, for comparison).
//
// In the multi-box form (erpp_batch_set_form), when every box runs the FP32
// step on x/y-halo tiles with compatible window variants and the fixed-point
// scatter, the graph instead holds nine launches for all boxes together: the
// binning (counts cleared, counted, scanned per box, records filled), ONE
// persistent gather over the (box, tile) work items of every box (densest
// boxes first, pulled from a counter), the advance of every particle, ONE
// persistent scatter, and the two halo merges.  Each phase then waits for
// every box's previous phase, where the branches let one box's binning
// overlap another's gather: on many small dense boxes the branches are the
// faster form (the binning's atomic increments of few tile counters, for
// one, are no longer hidden behind other boxes' work).
//
// The graph holds the descriptors' device pointers: the buffers must stay
// allocated and in place for the batch's lifetime (their contents change
// freely between steps).
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "erpp_internal.cuh"

struct erpp_batch {
  int32_t nbox;
  erpp_box_desc* boxes;
  erpp_ctx** ctx;
  cudaStream_t origin;
  cudaStream_t* branch;
  cudaEvent_t fork;
  cudaEvent_t* join;
  cudaGraphExec_t exec[2];  // [first_step]
  erpp::Multi4* multi;      // multi-box tile launches, or null
  int32_t form;             // ERPP_BATCH_BRANCHES or ERPP_BATCH_MULTI
};

namespace {

// Kernels of the multi-box step: clear, count, scan, fill, gather, advance,
// scatter, row merge, column merge.
constexpr int32_t kMultiLaunches = 9;

erpp_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ERPP_OK;
  if (e == cudaErrorMemoryAllocation) return ERPP_ENOMEM;
  return ERPP_ECUDA;
}

erpp_status capture(erpp_batch* b, int first_step) {
  if (!b->multi && b->form == ERPP_BATCH_MULTI) {
    // the multi-box launches need every box's scratch in place and the same
    // kernel variant; otherwise each box's own step is captured
    std::vector<erpp_ctx*> cs(b->ctx, b->ctx + b->nbox);
    if (erpp::multi4_eligible(cs.data(), b->nbox)) {
      std::vector<const float*> us((size_t)b->nbox);
      std::vector<float*> ss((size_t)b->nbox);
      std::vector<erpp_particles> ps((size_t)b->nbox);
      for (int i = 0; i < b->nbox; ++i) {
        us[(size_t)i] = (const float*)b->boxes[i].u;
        ss[(size_t)i] = (float*)b->boxes[i].S;
        ps[(size_t)i] = b->boxes[i].particles;
      }
      if (erpp::multi4_create(cs.data(), us.data(), ss.data(), ps.data(), b->nbox, &b->multi) !=
          cudaSuccess) {
        b->multi = nullptr;
        cudaGetLastError();
      }
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_status(e);
  erpp_status s = ERPP_OK;
  if (b->multi) {
    // one stream: binning, gather, advance, scatter and merges of all boxes
    for (int i = 0; i < b->nbox; ++i) b->ctx[i]->last_step_launches = 0;
    e = erpp::multi4_step(b->multi, first_step, b->origin);
  } else {
    e = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < b->nbox && e == cudaSuccess && s == ERPP_OK; ++i) {
      e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
      if (e != cudaSuccess) break;
      const erpp_box_desc& d = b->boxes[i];
      s = erpp_step(b->ctx[i], d.u, &d.particles, d.S, first_step, (erpp_stream)b->branch[i]);
      if (s != ERPP_OK) break;
      e = cudaEventRecord(b->join[i], b->branch[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
  }
  // always end the capture (a failed capture is discarded)
  cudaError_t e2 = cudaStreamEndCapture(b->origin, &graph);
  if (s == ERPP_OK && e == cudaSuccess) e = e2;
  if (s == ERPP_OK && e == cudaSuccess)
    e = cudaGraphInstantiateWithFlags(&b->exec[first_step], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (s != ERPP_OK) {
    cudaGetLastError();
    return s;
  }
  if (e != cudaSuccess) {
    b->exec[first_step] = nullptr;
    cudaGetLastError();
    return ERPP_ECUDA;
  }
  return ERPP_OK;
}

}  // namespace

extern "C" {

erpp_status erpp_batch_destroy(erpp_batch* b) {
  if (!b) return ERPP_OK;
  cudaDeviceSynchronize();
  for (int k = 0; k < 2; ++k)
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  erpp::multi4_destroy(b->multi);
  if (b->ctx)
    for (int i = 0; i < b->nbox; ++i) erpp_destroy(b->ctx[i]);
  if (b->branch)
    for (int i = 0; i < b->nbox; ++i)
      if (b->branch[i]) cudaStreamDestroy(b->branch[i]);
  if (b->join)
    for (int i = 0; i < b->nbox; ++i)
      if (b->join[i]) cudaEventDestroy(b->join[i]);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  free(b->ctx);
  free(b->branch);
  free(b->join);
  free(b->boxes);
  free(b);
  return ERPP_OK;
}

erpp_status erpp_batch_init(int32_t nbox, const erpp_box_desc* boxes, erpp_batch** out) {
  if (!out) return ERPP_EINVAL;
  *out = nullptr;
  if (nbox < 1 || nbox > ERPP_MAX_BOXES || !boxes) return ERPP_EINVAL;
  for (int i = 0; i < nbox; ++i) {
    const erpp_box_desc& d = boxes[i];
    const erpp_particles& P = d.particles;
    if (!d.u || !d.S || P.n < 0 || P.n > ERPP_MAX_PARTICLES) return ERPP_EINVAL;
    if (d.params.flags & (ERPP_PIC | ERPP_POINT_GATHER | ERPP_LAG | ERPP_FULL_FORCE))
      return ERPP_EINVAL;
    if (P.n > 0) {
      if (!P.radius || !P.rho_p) return ERPP_EINVAL;
      for (int a = 0; a < 3; ++a)
        if (!P.x[a] || !P.v[a] || !P.x_prev[a] || !P.D[a]) return ERPP_EINVAL;
    }
  }
  erpp_batch* b = (erpp_batch*)calloc(1, sizeof(erpp_batch));
  if (!b) return ERPP_ENOMEM;
  b->nbox = nbox;
  b->boxes = (erpp_box_desc*)malloc(sizeof(erpp_box_desc) * (size_t)nbox);
  b->ctx = (erpp_ctx**)calloc((size_t)nbox, sizeof(erpp_ctx*));
  b->branch = (cudaStream_t*)calloc((size_t)nbox, sizeof(cudaStream_t));
  b->join = (cudaEvent_t*)calloc((size_t)nbox, sizeof(cudaEvent_t));
  if (!b->boxes || !b->ctx || !b->branch || !b->join) {
    erpp_batch_destroy(b);
    return ERPP_ENOMEM;
  }
  memcpy(b->boxes, boxes, sizeof(erpp_box_desc) * (size_t)nbox);
  erpp_status s = ERPP_OK;
  for (int i = 0; i < nbox && s == ERPP_OK; ++i) {
    s = erpp_init(&b->boxes[i].params, &b->ctx[i]);
    // scratch for the box's particles now: no allocation may happen while
    // the step is being captured
    if (s == ERPP_OK) s = erpp::ensure_capacity(b->ctx[i], b->boxes[i].particles.n);
  }
  cudaError_t e = cudaSuccess;
  if (s == ERPP_OK) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (s == ERPP_OK && e == cudaSuccess)
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < nbox && s == ERPP_OK && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (s == ERPP_OK && e != cudaSuccess) s = cuda_status(e);
  if (s != ERPP_OK) {
    erpp_batch_destroy(b);
    cudaGetLastError();
    return s;
  }
  *out = b;
  return ERPP_OK;
}

erpp_status erpp_step_batched(erpp_batch* b, int first_step, int use_graph, erpp_stream stream) {
  if (!b) return ERPP_EINVAL;
  const int fs = first_step ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (!use_graph) {
    for (int i = 0; i < b->nbox; ++i) {
      const erpp_box_desc& d = b->boxes[i];
      erpp_status s = erpp_step(b->ctx[i], d.u, &d.particles, d.S, fs, stream);
      if (s != ERPP_OK) return s;
    }
    return ERPP_OK;
  }
  if (!b->exec[fs]) {
    // the capture streams must not start before the caller's prior work:
    // capture itself launches nothing, and each replay is ordered on `st`
    erpp_status s = capture(b, fs);
    if (s != ERPP_OK) return s;
  }
  return cuda_status(cudaGraphLaunch(b->exec[fs], st));
}

erpp_status erpp_batch_set_tiling(erpp_batch* b, int32_t box, int32_t tile_y, int32_t tile_z,
                                  int32_t threads) {
  if (!b || box < 0 || box >= b->nbox) return ERPP_EINVAL;
  erpp_status s = erpp_set_tiling(b->ctx[box], tile_y, tile_z, threads);
  // scratch again now (never during a capture), and the graphs hold the old
  // launch configuration
  if (s == ERPP_OK) s = erpp::ensure_capacity(b->ctx[box], b->boxes[box].particles.n);
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    b->exec[k] = nullptr;
  }
  // the multi-box descriptors hold the old scratch and tile shape
  cudaDeviceSynchronize();
  erpp::multi4_destroy(b->multi);
  b->multi = nullptr;
  return s;
}

erpp_status erpp_batch_set_form(erpp_batch* b, int32_t form) {
  if (!b || (form != ERPP_BATCH_BRANCHES && form != ERPP_BATCH_MULTI)) return ERPP_EINVAL;
  if (form == b->form) return ERPP_OK;
  b->form = form;
  cudaDeviceSynchronize();
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    b->exec[k] = nullptr;
  }
  erpp::multi4_destroy(b->multi);
  b->multi = nullptr;
  return ERPP_OK;
}

erpp_status erpp_batch_get_tiling(erpp_batch* b, int32_t box, int32_t out[5]) {
  if (!b || !out || box < 0 || box >= b->nbox) return ERPP_EINVAL;
  return erpp_get_tiling(b->ctx[box], out);
}

erpp_status erpp_batch_last_step_launches(erpp_batch* b, int32_t* n) {
  if (!b || !n) return ERPP_EINVAL;
  int32_t total = b->multi ? kMultiLaunches : 0;  // the multi-box step's kernels
  for (int i = 0; i < b->nbox; ++i) {
    int32_t k = 0;
    erpp_last_step_launches(b->ctx[i], &k);
    total += k;
  }
  *n = total;
  return ERPP_OK;
}

erpp_status erpp_batch_check(erpp_batch* b, erpp_stream stream) {
  if (!b) return ERPP_EINVAL;
  erpp_status worst = ERPP_OK;
  for (int i = 0; i < b->nbox; ++i) {
    erpp_status s = erpp_check(b->ctx[i], stream);
    if (s != ERPP_OK && worst == ERPP_OK) worst = s;
  }
  return worst;
}

}  // extern "C"
