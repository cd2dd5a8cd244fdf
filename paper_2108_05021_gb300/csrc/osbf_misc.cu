// Small elementwise kernels of the library (type conversion, fills).
#include "osbf_internal.h"

namespace osbf {

__global__ void u8_to_f32_kernel(const uint8_t *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void fill_u8_kernel(uint8_t *__restrict__ p, uint8_t v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// A synthetic image for tuning: 64 x 64 blocks of hashed levels in [0, 1] plus hashed
// noise of amplitude 0.05, clamped (values only need to be non-constant and image-like:
// the filter's cost does not depend on them, but a constant image would let every
// selection tie).  8-bit storage gets round(255 v).
__device__ __forceinline__ float hash01(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return (x >> 8) * (1.0f / 16777216.0f);
}

template <typename T>
__global__ void tuning_image_kernel(T *__restrict__ p, int H, int W, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long plane = i / ((long long)H * W);
        const int rem = (int)(i - plane * H * (long long)W), y = rem / W, x = rem - y * W;
        const unsigned cell = (unsigned)(plane * 7919 + (y >> 6) * 104729 + (x >> 6));
        float v = hash01(cell * 2654435761u) + 0.1f * (hash01((unsigned)i * 2246822519u + 7u) - 0.5f);
        v = fminf(fmaxf(v, 0.f), 1.f);
        if constexpr (sizeof(T) == 1)
            p[i] = (T)__float2int_rn(255.f * v);
        else
            p[i] = from_f<T>(v);
    }
}

static int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

cudaError_t launch_u8_to_f32(const uint8_t *in, float *out, long long n, cudaStream_t s) {
    u8_to_f32_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_tuning_image(Storage st, void *p, int P, int H, int W, cudaStream_t s) {
    const long long n = (long long)P * H * W;
    switch (st) {
    case Storage::F32: tuning_image_kernel<float><<<grid_for(n), 256, 0, s>>>((float *)p, H, W, n); break;
    case Storage::F16: tuning_image_kernel<__half><<<grid_for(n), 256, 0, s>>>((__half *)p, H, W, n); break;
    case Storage::BF16:
        tuning_image_kernel<__nv_bfloat16><<<grid_for(n), 256, 0, s>>>((__nv_bfloat16 *)p, H, W, n);
        break;
    case Storage::U8: tuning_image_kernel<uint8_t><<<grid_for(n), 256, 0, s>>>((uint8_t *)p, H, W, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_u8(uint8_t *p, uint8_t v, long long n, cudaStream_t s) {
    fill_u8_kernel<<<grid_for(n), 256, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

size_t fwd_smem(Storage st, int R, int D) {
    switch (st) {
    case Storage::F32: return fwd_smem_bytes<float, float>(R, D);
    case Storage::F16: return fwd_smem_bytes<__half, __half>(R, D);
    case Storage::BF16: return fwd_smem_bytes<__nv_bfloat16, __nv_bfloat16>(R, D);
    case Storage::U8: return fwd_smem_bytes<uint8_t, float>(R, D);
    }
    return 0;
}

}  // namespace osbf

// ------------------------------------------------------------------------------------
// the appendix's replicate padding: frame(fy, fx) = in(clamp(fy - R), clamp(fx - R))
// ------------------------------------------------------------------------------------
namespace osbf {

template <typename T>
__global__ void pad_replicate_kernel(const T *__restrict__ in, T *__restrict__ frame, int H, int W, int R, int FW,
                                     int FWp) {
    const int fy = blockIdx.y, plane = blockIdx.z;
    const int y = min(max(fy - R, 0), H - 1);
    const T *src = in + ((long long)plane * H + y) * W;
    T *dst = frame + ((long long)plane * gridDim.y + fy) * FWp;
    for (int fx = blockIdx.x * blockDim.x + threadIdx.x; fx < FW; fx += gridDim.x * blockDim.x)
        dst[fx] = src[min(max(fx - R, 0), W - 1)];
}

cudaError_t launch_pad_replicate(Storage st, const void *in, void *frame, int P, int H, int W, int R, int FH, int FW,
                                 int FWp, cudaStream_t s) {
    dim3 grid((FW + 255) / 256 < 8 ? (FW + 255) / 256 : 8, FH, P);
    switch (st) {
    case Storage::F32:
        pad_replicate_kernel<float><<<grid, 256, 0, s>>>((const float *)in, (float *)frame, H, W, R, FW, FWp);
        break;
    case Storage::F16:
        pad_replicate_kernel<__half><<<grid, 256, 0, s>>>((const __half *)in, (__half *)frame, H, W, R, FW, FWp);
        break;
    case Storage::BF16:
        pad_replicate_kernel<__nv_bfloat16>
            <<<grid, 256, 0, s>>>((const __nv_bfloat16 *)in, (__nv_bfloat16 *)frame, H, W, R, FW, FWp);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace osbf

namespace osbf {

// The appendix's final crop: frame rows/columns r .. r+H-1 / r .. r+W-1 into the output
// (E: the storage element; 16-bit values are copied as they are).
template <typename E>
__global__ void crop_kernel(const E *__restrict__ frame, E *__restrict__ out, int H, int W, int R, int FH, int FWp) {
    const int y = blockIdx.y, plane = blockIdx.z;
    const E *src = frame + ((long long)plane * FH + y + R) * FWp + R;
    E *dst = out + ((long long)plane * H + y) * W;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) dst[x] = src[x];
}

template <typename E>
static cudaError_t launch_crop(const E *frame, E *out, int P, int H, int W, int R, int FWp, cudaStream_t s) {
    for (int p0 = 0; p0 < P; p0 += 65535) {
        const int np = P - p0 < 65535 ? P - p0 : 65535;
        dim3 grid((W + 255) / 256 < 8 ? (W + 255) / 256 : 8, H, np);
        crop_kernel<E><<<grid, 256, 0, s>>>(frame + (size_t)p0 * (H + 2 * R) * FWp, out + (size_t)p0 * H * W, H, W, R,
                                            H + 2 * R, FWp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_crop_f32(const float *frame, float *out, int P, int H, int W, int R, int FWp, cudaStream_t s) {
    return launch_crop<float>(frame, out, P, H, W, R, FWp, s);
}

cudaError_t launch_crop_16(const void *frame, void *out, int P, int H, int W, int R, int FWp, cudaStream_t s) {
    return launch_crop<uint16_t>(static_cast<const uint16_t *>(frame), static_cast<uint16_t *>(out), P, H, W, R, FWp,
                                 s);
}

}  // namespace osbf
