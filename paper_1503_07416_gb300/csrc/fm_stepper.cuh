// Host driver of one time step, shared by the solvers of libfm.
//
// A solver Impl issues its step in three parts (static member functions):
//   enqueue_prepare(st)                          the explicit inputs of the step,
//   enqueue_resid_norm(st, in_body, hdl, use_h)  the float64 residual, its norm
//                                                and the control-block update,
//   enqueue_body(st, hdl, use_h)                 one cycle, the float64 update and
//                                                enqueue_resid_norm(st, 1, ...),
//   enqueue_post(st)                             the closure and commit of the new
//                                                time level (skipped on failure),
//                                                the control block to pinned memory;
// and Impl::NVEL, the velocity arrays of the state that step_host copies.
// Graph mode captures prepare, a WHILE conditional node around the body and
// post into one CUDA graph (one launch and one host synchronisation per
// step); host-loop mode (profiling) launches the parts directly and reads the
// control block after each norm.
#pragma once

#include <cuda_runtime.h>
#include <cstring>

#include "fm_state.h"
#include "fm_device.cuh"

#define FM_CUDA(call)                                   \
  do {                                                  \
    cudaError_t err__ = (call);                         \
    if (err__ != cudaSuccess) return FM_ECUDA;          \
  } while (0)

#define FM_LAUNCHED()                                   \
  do {                                                  \
    ++st->launches;                                     \
    if (cudaPeekAtLastError() != cudaSuccess) {         \
      cudaGetLastError();                               \
      return FM_ECUDA;                                  \
    }                                                   \
  } while (0)

namespace fm {

// Sum the durations of the recorded (start, end) event pairs; call only after
// the stream has been synchronised.
static inline int harvest_profile(fm_state* st) {
  for (int i = 0; i + 1 < st->npev; i += 2) {
    float ms = 0.f;
    FM_CUDA(cudaEventElapsedTime(&ms, st->pev[i], st->pev[i + 1]));
    st->prof_ms += ms;
    st->prof_count += 1;
  }
  st->npev = 0;
  return FM_OK;
}

template <class Impl>
struct Stepper {
  static int read_ctl(fm_state* st, Ctl* out) {
    FM_CUDA(cudaMemcpyAsync(st->hscal + 32, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    memcpy(out, st->hscal + 32, sizeof(Ctl));
    return harvest_profile(st);
  }

  static int finish(fm_state* st, fm_step_info* info) {
    Ctl c;
    memcpy(&c, st->hscal + 32, sizeof(Ctl));
    st->prepared = false;
    if (info) {
      info->cycles = c.cycles;
      info->res0 = c.norm0;
      info->res = c.norm;
    }
    return c.status;
  }

  static int step_hostloop(fm_state* st, fm_step_info* info) {
    int rc = Impl::enqueue_prepare(st);
    if (rc) return rc;
    rc = Impl::enqueue_resid_norm(st, 0, 0, 0);
    if (rc) return rc;
    Ctl c;
    for (;;) {
      rc = read_ctl(st, &c);
      if (rc) return rc;
      if (c.status != FM_OK || !(c.norm > st->prm.tol)) break;
      rc = Impl::enqueue_body(st, 0, 0);
      if (rc) return rc;
    }
    rc = Impl::enqueue_post(st);
    if (rc) return rc;
    FM_CUDA(cudaStreamSynchronize(st->stream));
    return finish(st, info);
  }

  static int build_graph(fm_state* st) {
    if (st->gexec) {
      cudaGraphExecDestroy(st->gexec);
      st->gexec = nullptr;
    }
    if (st->graph) {
      cudaGraphDestroy(st->graph);
      st->graph = nullptr;
    }
    cudaStream_t saved = st->stream;
    cudaStream_t s0 = st->cap[0], s1 = st->cap[1];
    st->capturing = true;
    st->stream = s0;
    int rc = FM_OK;
    cudaGraph_t g = nullptr;
    do {
      if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      const long long l0 = st->launches;
      rc = Impl::enqueue_prepare(st);
      if (rc) break;
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaGraph_t cg = nullptr;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphConditionalHandle hdl;
      if (cudaGraphConditionalHandleCreate(&hdl, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) { rc = FM_ECUDA; break; }
      rc = Impl::enqueue_resid_norm(st, 0, hdl, 1);
      if (rc) break;
      st->cnt_pre = st->launches - l0;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = hdl;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode;
      if (cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      if (cudaStreamUpdateCaptureDependencies(s0, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) { rc = FM_ECUDA; break; }
      st->stream = s1;
      if (cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      const long long l1 = st->launches;
      rc = Impl::enqueue_body(st, hdl, 1);
      st->cnt_body = st->launches - l1;
      cudaGraph_t bodyout = nullptr;
      if (cudaStreamEndCapture(s1, &bodyout) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
      if (rc) break;
      st->stream = s0;
      const long long l2 = st->launches;
      rc = Impl::enqueue_post(st);
      st->cnt_post = st->launches - l2;
      st->launches = l0;
    } while (0);
    st->stream = s0;
    if (cudaStreamEndCapture(s0, &g) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
    st->stream = saved;
    st->capturing = false;
    if (rc) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (cudaGraphInstantiate(&st->gexec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      return FM_ECUDA;
    }
    st->graph = g;
    st->graph_dt = st->dt;
    return FM_OK;
  }

  // One step for host-resident fields: the input copies, the step and the
  // output copies on the state's stream, one host synchronisation (graph
  // mode).  On failure the state and the outputs keep time level k.
  static int step_host(fm_state* st, const double* rho_in, const double* const* vel_in, double* rho_out,
                       double* const* vel_out, fm_step_info* info) {
    const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
    const bool graph = !(st->prof || !st->use_graph);
    if (graph && (!st->gexec || st->graph_dt != st->dt)) {
      const int rc = build_graph(st);  // captured on private streams
      if (rc) return rc;
    }
    FM_CUDA(cudaMemcpyAsync(st->rho, rho_in, bytes, cudaMemcpyHostToDevice, st->stream));
    for (int d = 0; d < Impl::NVEL; ++d)
      FM_CUDA(cudaMemcpyAsync(st->vel[d], vel_in[d], bytes, cudaMemcpyHostToDevice, st->stream));
    st->prepared = false;
    int rc;
    if (graph) {
      FM_CUDA(cudaGraphLaunch(st->gexec, st->stream));
      rc = FM_OK;
    } else {
      rc = step_hostloop(st, nullptr);  // synchronises; status read below
      if (rc != FM_OK && rc != FM_ENOCONV && rc != FM_ENAN && rc != FM_ENONPOS) return rc;
    }
    FM_CUDA(cudaMemcpyAsync(rho_out, st->rho, bytes, cudaMemcpyDeviceToHost, st->stream));
    for (int d = 0; d < Impl::NVEL; ++d)
      FM_CUDA(cudaMemcpyAsync(vel_out[d], st->vel[d], bytes, cudaMemcpyDeviceToHost, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    if (graph) {
      Ctl c;
      memcpy(&c, st->hscal + 32, sizeof(Ctl));
      st->launches += st->cnt_pre + (long long)c.cycles * st->cnt_body + st->cnt_post;
    }
    return finish(st, info);
  }

  static int step(fm_state* st, fm_step_info* info) {
    if (st->prof || !st->use_graph) return step_hostloop(st, info);
    if (!st->gexec || st->graph_dt != st->dt) {
      int rc = build_graph(st);
      if (rc) return rc;
    }
    FM_CUDA(cudaGraphLaunch(st->gexec, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    Ctl c;
    memcpy(&c, st->hscal + 32, sizeof(Ctl));
    st->launches += st->cnt_pre + (long long)c.cycles * st->cnt_body + st->cnt_post;
    return finish(st, info);
  }
};

}  // namespace fm
