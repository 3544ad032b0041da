// rhd_host.cuh -- the update of a grid whose state lives in host memory.
//
// The cells go through the GPU in chunks.  Three device staging sets rotate:
// while chunk k is solved on the compute stream, chunk k+1 is copied in on one
// copy stream and chunk k-1 copied out on another (the two directions use
// separate copy engines), so the transfers hide behind the solve.  Events
// order the three streams: a set is refilled only after the copy-out that
// last read it, a chunk is solved only after its copy-in, and copied out only
// after its solve.  Per-group arrays move as 2-D copies (N_g rows of the
// chunk's cells, host pitch = the host group stride).  Each chunk is one
// ordinary rhd_source_update / rhd_source_update_warm call on the staging
// set, so the results are those of the device entry, cell for cell.
#pragma once

namespace rhd {
namespace {

constexpr int kHostSets = 3;
constexpr int64_t kHostChunk = 1 << 20;

struct HostPipe {
  bool init = false;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t in_done[kHostSets], comp_done[kHostSets], out_done[kHostSets];
  char *buf = nullptr;
  size_t set_bytes = 0;
};
HostPipe g_host[kMaxDevices];

// Staging set layout for m cells and G groups (all FP64 unless noted):
// rho, egas, kappa0 [m]; mom [3][m]; erad, src [G][m]; frad [3][G][m];
// status, iters [m] bytes.
size_t host_set_bytes(int64_t m, int G) {
  return (size_t)m * 8 * (3 + 3 + 2 * (size_t)G + 3 * (size_t)G) + 2 * (size_t)m + 256;
}

int host_pipe(int dev, size_t set_bytes, HostPipe **out) {
  HostPipe &p = g_host[dev];
  if (!p.init) {
    if (cudaStreamCreateWithFlags(&p.s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p.s_comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p.s_out, cudaStreamNonBlocking) != cudaSuccess)
      return RHD_ECUDA;
    for (int s = 0; s < kHostSets; ++s)
      if (cudaEventCreateWithFlags(&p.in_done[s], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p.comp_done[s], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p.out_done[s], cudaEventDisableTiming) != cudaSuccess)
        return RHD_ECUDA;
    p.init = true;
  }
  if (p.set_bytes < set_bytes) {
    if (p.buf) {
      cudaDeviceSynchronize();
      cudaFree(p.buf);
      p.buf = nullptr;
      p.set_bytes = 0;
    }
    if (cudaMalloc(&p.buf, set_bytes * kHostSets) != cudaSuccess) return RHD_ENOMEM;
    p.set_bytes = set_bytes;
  }
  *out = &p;
  return RHD_OK;
}

// Device state of staging set s for m cells (group stride m), pointers into buf.
rhd_state_t host_set_state(const rhd_state_t &h, char *base, int64_t m, int G) {
  rhd_state_t d = h;
  double *p = reinterpret_cast<double *>(base);
  d.rho = p;
  p += m;
  d.egas = p;
  p += m;
  double *k0 = p;
  p += m;
  d.kappa0 = h.kappa0 ? k0 : nullptr;
  for (int c = 0; c < 3; ++c, p += m) d.mom[c] = p;
  d.erad = p;
  p += (int64_t)G * m;
  double *src = p;
  p += (int64_t)G * m;
  d.src = h.src ? src : nullptr;
  for (int c = 0; c < 3; ++c, p += (int64_t)G * m) d.frad[c] = p;
  uint8_t *b = reinterpret_cast<uint8_t *>(p);
  d.status = h.status ? b : nullptr;
  d.iters = h.iters ? b + m : nullptr;
  d.group_stride = 0;  // = m
  return d;
}

cudaError_t copy_rows(void *dst, int64_t dpitch, const void *src, int64_t spitch, int64_t width,
                      int64_t rows, cudaMemcpyKind kind, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, (size_t)dpitch, src, (size_t)spitch, (size_t)width, (size_t)rows,
                           kind, st);
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_source_update_host(rhd_state_t *state, const rhd_groups_t *groups,
                                      const rhd_opacity_law_t *opacity_law, double dt,
                                      int64_t n_cells, rhd_surrogate_t *surrogate,
                                      int64_t chunk_cells) {
  using namespace rhd;
  if (!state || !groups || n_cells < 0 || chunk_cells < 0) return RHD_EINVAL;
  {  // every argument check of the device entry, on the host state
    static thread_local KParams kp;
    const int rc = pack(state, groups, opacity_law, dt, n_cells, &kp);
    if (rc != RHD_OK) return rc;
  }
  if (n_cells == 0) return RHD_OK;
  int sms = 0;
  int rc = ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RHD_ECUDA;
  const int G = groups->n_groups;
  const int64_t m_max = chunk_cells > 0 ? chunk_cells : kHostChunk;
  const int64_t hgs = state->group_stride ? state->group_stride : n_cells;
  HostPipe *p = nullptr;
  rc = host_pipe(dev, host_set_bytes(m_max, G), &p);
  if (rc != RHD_OK) return rc;
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
  const int64_t nchunks = (n_cells + m_max - 1) / m_max;
  for (int64_t k = 0; k < nchunks && rc == RHD_OK; ++k) {
    const int s = (int)(k % kHostSets);
    const int64_t c0 = k * m_max, m = n_cells - c0 < m_max ? n_cells - c0 : m_max;
    rhd_state_t d = host_set_state(*state, p->buf + (size_t)s * p->set_bytes, m, G);
    const int64_t b = m * 8;
    cudaError_t e = cudaSuccess;
    // ---- copy in (after the copy-out that last read this set)
    if (k >= kHostSets) e = cudaStreamWaitEvent(p->s_in, p->out_done[s], 0);
    auto in1 = [&](double *dst, const double *src) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src + c0, b, H2D, p->s_in);
    };
    auto inG = [&](double *dst, const double *src) {
      if (e == cudaSuccess) e = copy_rows(dst, b, src + c0, hgs * 8, b, G, H2D, p->s_in);
    };
    in1(const_cast<double *>(d.rho), state->rho);
    in1(d.egas, state->egas);
    if (state->kappa0) in1(const_cast<double *>(d.kappa0), state->kappa0);
    for (int c = 0; c < 3; ++c) in1(d.mom[c], state->mom[c]);
    inG(d.erad, state->erad);
    if (state->src) inG(const_cast<double *>(d.src), state->src);
    for (int c = 0; c < 3; ++c) inG(d.frad[c], state->frad[c]);
    if (e == cudaSuccess) e = cudaEventRecord(p->in_done[s], p->s_in);
    // ---- solve
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, p->in_done[s], 0);
    if (e != cudaSuccess) {
      rc = RHD_ECUDA;
      break;
    }
    rc = surrogate ? rhd_source_update_warm(surrogate, &d, groups, opacity_law, dt, m, p->s_comp)
                   : rhd_source_update(&d, groups, opacity_law, dt, m, p->s_comp);
    if (rc != RHD_OK) break;
    e = cudaEventRecord(p->comp_done[s], p->s_comp);
    // ---- copy out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, p->comp_done[s], 0);
    auto out1 = [&](double *dst, const double *src) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(dst + c0, src, b, D2H, p->s_out);
    };
    auto outG = [&](double *dst, const double *src) {
      if (e == cudaSuccess) e = copy_rows(dst + c0, hgs * 8, src, b, b, G, D2H, p->s_out);
    };
    out1(state->egas, d.egas);
    for (int c = 0; c < 3; ++c) out1(state->mom[c], d.mom[c]);
    outG(state->erad, d.erad);
    for (int c = 0; c < 3; ++c) outG(state->frad[c], d.frad[c]);
    if (state->status && e == cudaSuccess)
      e = cudaMemcpyAsync(state->status + c0, d.status, (size_t)m, D2H, p->s_out);
    if (state->iters && e == cudaSuccess)
      e = cudaMemcpyAsync(state->iters + c0, d.iters, (size_t)m, D2H, p->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(p->out_done[s], p->s_out);
    if (e != cudaSuccess) rc = RHD_ECUDA;
  }
  // every chunk's copies and solve end before the call returns (also after
  // an error, so that no transfer outlives the caller's buffers)
  const cudaError_t e1 = cudaStreamSynchronize(p->s_in);
  const cudaError_t e2 = cudaStreamSynchronize(p->s_comp);
  const cudaError_t e3 = cudaStreamSynchronize(p->s_out);
  if (rc == RHD_OK && (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)) rc = RHD_ECUDA;
  return rc;
}
