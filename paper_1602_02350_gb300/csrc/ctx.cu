// Context, scratch memory and error reporting of the C ABI.
#include "common.cuh"

static thread_local char g_err[1024] = "";

void rs_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int rs_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int rs_enter(rs_ctx* ctx) {
  if (!ctx) return rs_fail(RS_EINVAL, "null context");
  int cur = -1;
  RS_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != ctx->device) RS_CUDA_TRY(cudaSetDevice(ctx->device));
  ++ctx->call_gen;
  return RS_OK;
}

void* rs_scratch(rs_ctx* ctx, int slot, size_t bytes) {
  ScratchSlot& s = ctx->slots[slot];
  if (bytes == 0) bytes = 16;
  if (s.bytes >= bytes) return s.ptr;
  if (s.ptr) {
    // the old buffer may still be read by queued work
    cudaStreamSynchronize(ctx->stream);
    cudaFree(s.ptr);
    s.ptr = nullptr;
    s.bytes = 0;
  }
  size_t want = bytes + bytes / 8;   // grow with slack to avoid repeated reallocations
  want = (want + 255) & ~size_t(255);
  if (cudaMalloc(&s.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    s.ptr = nullptr;
    rs_set_error("cudaMalloc of %zu bytes for scratch slot %d failed", want, slot);
    return nullptr;
  }
  s.bytes = want;
  return s.ptr;
}

int check_matrix(const rs_matrix* X, const char* name) {
  if (!X || !X->data) return rs_fail(RS_EINVAL, "%s: null matrix", name);
  if (X->n <= 0 || X->d <= 0 || X->ld < X->d)
    return rs_fail(RS_EINVAL, "%s: bad shape n=%lld d=%lld ld=%lld", name, (long long)X->n, (long long)X->d,
                   (long long)X->ld);
  if (dtype_size(X->dtype) == 0) return rs_fail(RS_EINVAL, "%s: bad dtype %d", name, X->dtype);
  if (!aligned16(X->data) || (X->ld * (int64_t)dtype_size(X->dtype)) % 16 != 0)
    return rs_fail(RS_EINVAL, "%s: base address and row stride must be multiples of 16 bytes", name);
  if (X->dtype == RS_FP8E4M3 && !X->row_scale) return rs_fail(RS_EINVAL, "%s: FP8 data needs row_scale", name);
  return RS_OK;
}

extern "C" {

const char* rs_last_error(void) { return g_err; }

int rs_abi_version(void) { return RS_ABI_VERSION; }

int rs_create(rs_ctx** out, int device, void* stream) {
  if (!out) return rs_fail(RS_EINVAL, "rs_create: null output pointer");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return rs_fail(RS_ECUDA, "rs_create: no CUDA device (%s)", cudaGetErrorString(e));
  }
  if (device < 0 || device >= count) return rs_fail(RS_EINVAL, "rs_create: device %d out of range", device);
  RS_CUDA_TRY(cudaSetDevice(device));
  rs_ctx* ctx = new rs_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete ctx;
    return rs_fail(RS_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  }
  ctx->num_sms = prop.multiProcessorCount;
  if (prop.major < 10) {
    delete ctx;
    return rs_fail(RS_EUNSUPPORTED, "rs_create: device %d is sm_%d%d; this library is built for sm_103a", device,
                   prop.major, prop.minor);
  }
  void* st = rs_scratch(ctx, SCR_STATUS, 16);
  if (!st) {
    delete ctx;
    return RS_ENOMEM;
  }
  ctx->d_status = static_cast<int*>(st);
  e = cudaMemsetAsync(ctx->d_status, 0, 16, ctx->stream);
  if (e != cudaSuccess) {
    delete ctx;
    return rs_fail(RS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  *out = ctx;
  return RS_OK;
}

int rs_destroy(rs_ctx* ctx) {
  if (!ctx) return RS_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& s : ctx->slots)
    if (s.ptr) cudaFree(s.ptr);
  delete ctx;
  return RS_OK;
}

int rs_set_stream(rs_ctx* ctx, void* stream) {
  if (!ctx) return rs_fail(RS_EINVAL, "null context");
  ctx->stream = static_cast<cudaStream_t>(stream);
  return RS_OK;
}

int64_t rs_launch_count(const rs_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
