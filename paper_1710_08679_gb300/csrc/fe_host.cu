// fe_ebe_apply_host: products with host-resident vectors, pipelined across calls.
//
// Call i uses buffer set k = i mod 2. Its copy-in (stream `in`) waits until the
// product of call i-2 has finished reading x[k]; its product (stream `comp`)
// waits for its copy-in and for the copy-out of call i-2 from y[k]; its copy-out
// (stream `out`) waits for its product; the caller's stream waits for the
// copy-out. Consecutive calls therefore overlap copy-in, product and copy-out.
#include "fe_internal.cuh"

namespace fe {

HostPipe::~HostPipe() {
  for (int k = 0; k < 2; ++k) {
    if (h2d[k]) cudaEventDestroy(h2d[k]);
    if (done[k]) cudaEventDestroy(done[k]);
    if (d2h[k]) cudaEventDestroy(d2h[k]);
  }
  if (in) cudaStreamDestroy(in);
  if (comp) cudaStreamDestroy(comp);
  if (out) cudaStreamDestroy(out);
}

namespace {

HostPipe& host_pipe(fe_mesh* m, int R, fe_dtype dtype) {
  std::unique_ptr<HostPipe>& hp = m->host_pipe;
  if (hp && hp->R == R && hp->dtype == (int)dtype) return *hp;
  if (hp) FE_CUDA(cudaDeviceSynchronize());  // the old buffers may still be in use
  hp.reset(new HostPipe());
  hp->R = R;
  hp->dtype = (int)dtype;
  const size_t bytes = (size_t)m->n_nodes * R * 3 * (dtype == FE_F64 ? sizeof(double) : sizeof(float));
  for (int k = 0; k < 2; ++k) {
    hp->x[k].alloc(bytes);
    hp->y[k].alloc(bytes);
  }
  FE_CUDA(cudaStreamCreateWithFlags(&hp->in, cudaStreamNonBlocking));
  FE_CUDA(cudaStreamCreateWithFlags(&hp->comp, cudaStreamNonBlocking));
  FE_CUDA(cudaStreamCreateWithFlags(&hp->out, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    FE_CUDA(cudaEventCreateWithFlags(&hp->h2d[k], cudaEventDisableTiming));
    FE_CUDA(cudaEventCreateWithFlags(&hp->done[k], cudaEventDisableTiming));
    FE_CUDA(cudaEventCreateWithFlags(&hp->d2h[k], cudaEventDisableTiming));
    // start in the "previous use finished" state
    FE_CUDA(cudaEventRecord(hp->done[k], hp->comp));
    FE_CUDA(cudaEventRecord(hp->d2h[k], hp->out));
  }
  return *hp;
}

}  // namespace
}  // namespace fe

extern "C" fe_status fe_ebe_apply_host(fe_mesh* m, int32_t R, fe_dtype dtype, const void* x_host, void* y_host,
                                       void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    FE_REQUIRE(dtype == FE_F64 || dtype == FE_F32, "unknown dtype %d", (int)dtype);
    FE_REQUIRE(x_host != nullptr && y_host != nullptr, "NULL vector");
    FE_REQUIRE(x_host != y_host, "x and y must not alias");
    fe::DeviceGuard dg(m->device);
    fe::HostPipe& hp = fe::host_pipe(m, R, dtype);
    const int k = hp.next;
    hp.next ^= 1;
    const size_t bytes = hp.x[k].bytes;
    FE_CUDA(cudaStreamWaitEvent(hp.in, hp.done[k], 0));
    FE_CUDA(cudaMemcpyAsync(hp.x[k].ptr, x_host, bytes, cudaMemcpyHostToDevice, hp.in));
    FE_CUDA(cudaEventRecord(hp.h2d[k], hp.in));
    FE_CUDA(cudaStreamWaitEvent(hp.comp, hp.h2d[k], 0));
    FE_CUDA(cudaStreamWaitEvent(hp.comp, hp.d2h[k], 0));
    if (dtype == FE_F64)
      fe::ebe_apply<double>(m, R, hp.x[k].as<double>(), hp.y[k].as<double>(), hp.comp);
    else
      fe::ebe_apply<float>(m, R, hp.x[k].as<float>(), hp.y[k].as<float>(), hp.comp);
    FE_CUDA(cudaEventRecord(hp.done[k], hp.comp));
    FE_CUDA(cudaStreamWaitEvent(hp.out, hp.done[k], 0));
    FE_CUDA(cudaMemcpyAsync(y_host, hp.y[k].ptr, bytes, cudaMemcpyDeviceToHost, hp.out));
    FE_CUDA(cudaEventRecord(hp.d2h[k], hp.out));
    FE_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, hp.d2h[k], 0));
  });
}
