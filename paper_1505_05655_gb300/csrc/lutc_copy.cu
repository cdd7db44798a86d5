// Row copies between host and device memory driven by the SMs.
//
// A request's raster and output in host memory are strided (rows of a few KB
// with a pitch): copy engines move such 2-D copies row by row and fall far
// below the host link's bandwidth.  On GB300 page-locked host memory is
// addressable from kernels over NVLink-C2C, so a kernel that moves 16-byte
// vectors of every row (reads of host memory for copies in, writes for
// copies out) runs at the link's rate whatever the row length.
#include <stdint.h>

#include "lutc_internal.cuh"

namespace lutc {
namespace {

template <int E>
struct Vec;
template <> struct Vec<16> { using T = uint4; };
template <> struct Vec<8> { using T = uint2; };
template <> struct Vec<4> { using T = uint32_t; };
template <> struct Vec<2> { using T = uint16_t; };
template <> struct Vec<1> { using T = uint8_t; };

// rows of `width` bytes, moved in E-byte units (every address and pitch a multiple of E); a row's
// tail shorter than E is moved byte by byte
template <int E>
__global__ void __launch_bounds__(256) k_copy_rows(uint8_t* __restrict__ dst, int64_t dpitch,
                                                   const uint8_t* __restrict__ src, int64_t spitch, int64_t width,
                                                   int64_t rows)
{
    using T = typename Vec<E>::T;
    const int64_t per_row = (width + E - 1) / E;
    const int64_t total = per_row * rows;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t r = i / per_row, c = (i - r * per_row) * E;
        const uint8_t* s = src + r * spitch + c;
        uint8_t* d = dst + r * dpitch + c;
        if (c + E <= width) {
            *reinterpret_cast<T*>(d) = *reinterpret_cast<const T*>(s);
        } else {
            for (int64_t k = 0; c + k < width; ++k) d[k] = s[k];
        }
    }
}

int elem_of(const void* dst, int64_t dpitch, const void* src, int64_t spitch)
{
    const uint64_t bits = (uint64_t)(uintptr_t)dst | (uint64_t)(uintptr_t)src | (uint64_t)dpitch | (uint64_t)spitch;
    for (int e = 16; e > 1; e /= 2)
        if ((bits & (uint64_t)(e - 1)) == 0) return e;
    return 1;
}

}  // namespace

bool device_can_access(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
           a.devicePointer == p;
}

int copy_rows(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t width, int64_t rows,
              cudaStream_t st)
{
    if (width <= 0 || rows <= 0) return LUTC_OK;
    const int e = elem_of(dst, dpitch, src, spitch);
    const int64_t units = (width + e - 1) / e * rows;
    const int grid = (int)std::min<int64_t>((units + 255) / 256, (int64_t)sm_count() * 8);
    uint8_t* d = reinterpret_cast<uint8_t*>(dst);
    const uint8_t* s = reinterpret_cast<const uint8_t*>(src);
    switch (e) {
    case 16: k_copy_rows<16><<<grid, 256, 0, st>>>(d, dpitch, s, spitch, width, rows); break;
    case 8: k_copy_rows<8><<<grid, 256, 0, st>>>(d, dpitch, s, spitch, width, rows); break;
    case 4: k_copy_rows<4><<<grid, 256, 0, st>>>(d, dpitch, s, spitch, width, rows); break;
    case 2: k_copy_rows<2><<<grid, 256, 0, st>>>(d, dpitch, s, spitch, width, rows); break;
    default: k_copy_rows<1><<<grid, 256, 0, st>>>(d, dpitch, s, spitch, width, rows); break;
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace lutc
