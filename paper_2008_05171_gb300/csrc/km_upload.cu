// km_upload.cu -- kmedoids_upload_matrix / kmedoids_upload_rows: the
// dissimilarity matrix from host memory into the caller's device buffer, row
// by row from one row pitch to another, padding columns cleared.
//
// From page-locked (pinned or registered) host memory the rows are read by
// the SMs themselves, 16-byte loads over the CPU-GPU link into the device
// buffer.  On a GB300 this reads the link at its full rate on every call
// (about 210 GB/s from Grace memory), where copy-engine transfers of the
// same buffer took anywhere from that to a quarter of it.  Memory the device
// cannot address (plain pageable memory) goes through cudaMemcpy2DAsync.
#define KM_SRC_ID 12  // names this file in bounds-check reports
#include <cstdio>
#include <cstring>

#include "../../include/kmedoids.h"
#include "km_internal.h"

namespace km {
namespace {

constexpr int kUpThreads = 512;
constexpr int kUpUnroll = 4;

// One flat 16-byte copy (both pitches equal the row length, aligned).
__global__ void __launch_bounds__(kUpThreads) k_upload_flat(const uint4* __restrict__ src,
                                                            uint4* __restrict__ dst, size_t n16) {
  const size_t stride = (size_t)gridDim.x * kUpThreads;
  size_t i = (size_t)blockIdx.x * kUpThreads + threadIdx.x;
  // kUpUnroll loads in flight per thread before their stores
  for (; i + (kUpUnroll - 1) * stride < n16; i += kUpUnroll * stride) {
    uint4 v[kUpUnroll];
#pragma unroll
    for (int u = 0; u < kUpUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
    for (int u = 0; u < kUpUnroll; ++u) dst[i + u * stride] = v[u];
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

// Rows of row_bytes from src (pitch sp) to dst (pitch dp), the rest of each
// destination row (dp - row_bytes bytes) set to zero.  A block per row,
// rows strided over the grid; W is the access width the alignment of both
// pitches, both bases and row_bytes allows (16, 4 or 2 bytes).
template <class W>
__global__ void __launch_bounds__(kUpThreads) k_upload_rows(const unsigned char* __restrict__ src,
                                                            size_t sp, unsigned char* __restrict__ dst,
                                                            size_t dp, size_t row_bytes, long long rows) {
  const size_t nw = row_bytes / sizeof(W);
  const size_t pad = (dp - row_bytes) / 2;  // pad bytes, cleared 2 at a time
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const W* s = reinterpret_cast<const W*>(src + (size_t)r * sp);
    W* d = reinterpret_cast<W*>(dst + (size_t)r * dp);
    for (size_t j = threadIdx.x; j < nw; j += kUpThreads) d[j] = s[j];
    uint16_t* dz = reinterpret_cast<uint16_t*>(dst + (size_t)r * dp + row_bytes);
    for (size_t j = threadIdx.x; j < pad; j += kUpThreads) dz[j] = 0;
  }
}

km_status up_fail(km_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace
}  // namespace km

using namespace km;

extern "C" km_status kmedoids_upload_rows(const void* host, int64_t host_ld, int32_t dtype,
                                          int64_t rows, int64_t n, void* D, int64_t ld,
                                          void* stream) {
  set_last_error("");
  if (dtype != KM_I32 && dtype != KM_F32 && dtype != KM_U16)
    return up_fail(KM_E_INVALID, "dtype must be KM_I32, KM_F32 or KM_U16");
  if (!host || !D) return up_fail(KM_E_INVALID, "host and D must be non-NULL");
  if (rows <= 0 || n <= 0 || host_ld < n || ld < n)
    return up_fail(KM_E_INVALID, "need rows > 0, n > 0, host_ld >= n and ld >= n");
  const size_t es = dtype == KM_U16 ? 2 : 4;
  if ((double)rows * (double)(ld > host_ld ? ld : host_ld) * (double)es > 0x1p60)
    return up_fail(KM_E_INVALID, "matrix too large");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = (size_t)n * es, sp = (size_t)host_ld * es, dp = (size_t)ld * es;
  char buf[256];

  cudaPointerAttributes pa;
  memset(&pa, 0, sizeof(pa));
  cudaError_t e = cudaPointerGetAttributes(&pa, host);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    pa.type = cudaMemoryTypeUnregistered;
  }
  if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)
    return up_fail(KM_E_INVALID, "host is a device address (use cudaMemcpy2DAsync)");
  const unsigned char* src = static_cast<const unsigned char*>(pa.devicePointer);
  if (pa.type == cudaMemoryTypeHost && src) {
    // the last byte read must lie in page-locked memory too, at the same
    // offset of the device mapping
    const size_t last = (size_t)(rows - 1) * sp + row - 1;
    cudaPointerAttributes pb;
    memset(&pb, 0, sizeof(pb));
    if (cudaPointerGetAttributes(&pb, static_cast<const unsigned char*>(host) + last) != cudaSuccess) {
      (void)cudaGetLastError();
      src = nullptr;
    } else if (pb.type != cudaMemoryTypeHost ||
               static_cast<const unsigned char*>(pb.devicePointer) != src + last) {
      src = nullptr;
    }
  }
  if (pa.type != cudaMemoryTypeHost || !src) {
    // not addressable by the device: the copy engines, then the pad columns
    e = cudaMemcpy2DAsync(D, dp, host, sp, row, (size_t)rows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && dp > row)
      e = cudaMemset2DAsync(static_cast<char*>(D) + row, dp, 0, dp - row, (size_t)rows, s);
  } else {
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
      unsigned char* dst = static_cast<unsigned char*>(D);
      const uintptr_t al = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
      if (sp == row && dp == row && (al % 16) == 0 && ((size_t)rows * row) % 16 == 0) {
        const size_t n16 = (size_t)rows * row / 16;
        k_upload_flat<<<sms * 4, kUpThreads, 0, s>>>(reinterpret_cast<const uint4*>(src),
                                                      reinterpret_cast<uint4*>(dst), n16);
      } else {
        const int grid = (int)(rows < (int64_t)sms * 8 ? rows : (int64_t)sms * 8);
        const size_t mix = al | sp | dp | row;
        if (mix % 16 == 0)
          k_upload_rows<uint4><<<grid, kUpThreads, 0, s>>>(src, sp, dst, dp, row, rows);
        else if (mix % 4 == 0)
          k_upload_rows<uint32_t><<<grid, kUpThreads, 0, s>>>(src, sp, dst, dp, row, rows);
        else
          k_upload_rows<uint16_t><<<grid, kUpThreads, 0, s>>>(src, sp, dst, dp, row, rows);
      }
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    set_last_error(buf);
    return KM_E_CUDA;
  }
  return KM_OK;
}

extern "C" km_status kmedoids_upload_matrix(const void* host, int64_t host_ld, int32_t dtype,
                                            int64_t n, void* D, int64_t ld, void* stream) {
  return kmedoids_upload_rows(host, host_ld, dtype, n, n, D, ld, stream);
}
