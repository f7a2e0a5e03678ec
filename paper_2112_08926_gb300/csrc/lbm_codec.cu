// Device-array entry points of the 16-bit storage codecs (Sec. 3): the same
// device functions the stream-collide kernels use for load and store.
#include <functional>

#include "lbm.h"
#include "lbm_device.cuh"

using namespace lbm;

namespace {

template <int FMT>
__global__ void k_encode(const float* __restrict__ x, uint16_t* __restrict__ out, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (uint16_t)Codec16<FMT>::enc(x[t]);
}

template <int FMT>
__global__ void k_decode(const uint16_t* __restrict__ c, float* __restrict__ out, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = Codec16<FMT>::dec(c[t]);
}

template <int FMT>
__global__ void k_encode_bits(uint32_t first, uint16_t* __restrict__ out, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (uint16_t)Codec16<FMT>::enc(__uint_as_float(first + (uint32_t)t));
}

// the table-driven posit encoder of the paired stream-collide kernel, on the
// same shared-memory copy of the table (x scaled by 2^SL as the kernel's
// values are; NaN keeps the sign of x)
template <int FMT>
__global__ void k_encode_bits_table(uint32_t first, uint16_t* __restrict__ out, int64_t n) {
    __shared__ EncEntry tab[512];
    for (int i = threadIdx.x; i < 512; i += blockDim.x) tab[i] = kEncTable<FMT>.e[i];
    __syncthreads();
    constexpr int SL = Codec16<FMT>::SL;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float x = __uint_as_float(first + (uint32_t)t);
        const uint32_t c = SL == 0 ? enc_table(tab, x)
                                   : (enc_table(tab, fabsf(x) * 128.0f) | ((__float_as_uint(x) >> 16) & 0x8000u));
        out[t] = (uint16_t)c;
    }
}

unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 64 ? (b > 0 ? b : 1) : 152 * 64);
}

template <template <int> class K, class... Args>
lbm_status dispatch(int storage, int64_t n, cudaStream_t s, Args... args) {
    if (n < 0) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
    const unsigned g = grid_for(n);
    switch (storage) {
    case LBM_FP16:   K<LBM_FP16>::run(g, s, args...); break;
    case LBM_FP16S:  K<LBM_FP16S>::run(g, s, args...); break;
    case LBM_FP16C:  K<LBM_FP16C>::run(g, s, args...); break;
    case LBM_P16_0S: K<LBM_P16_0S>::run(g, s, args...); break;
    case LBM_P16_1S: K<LBM_P16_1S>::run(g, s, args...); break;
    case LBM_P16_2C: K<LBM_P16_2C>::run(g, s, args...); break;
    case LBM_P16_0:  K<LBM_P16_0>::run(g, s, args...); break;
    case LBM_P16_1:  K<LBM_P16_1>::run(g, s, args...); break;
    default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int F> struct Enc {
    static void run(unsigned g, cudaStream_t s, const float* x, uint16_t* o, int64_t n) {
        k_encode<F><<<g, 256, 0, s>>>(x, o, n);
    }
};
template <int F> struct Dec {
    static void run(unsigned g, cudaStream_t s, const uint16_t* c, float* o, int64_t n) {
        k_decode<F><<<g, 256, 0, s>>>(c, o, n);
    }
};
template <int F> struct EncBits {
    static void run(unsigned g, cudaStream_t s, uint32_t first, uint16_t* o, int64_t n) {
        k_encode_bits<F><<<g, 256, 0, s>>>(first, o, n);
    }
};

template <int F> struct EncBitsTable {
    static void run(unsigned g, cudaStream_t s, uint32_t first, uint16_t* o, int64_t n) {
        k_encode_bits_table<F><<<g, 256, 0, s>>>(first, o, n);
    }
};

}  // namespace

extern "C" {

lbm_status lbm_codec_encode(int storage, const float* x_dev, uint16_t* out_dev, int64_t n, void* stream) {
    if (n > 0 && (!x_dev || !out_dev)) return LBM_ERR_ARG;
    return dispatch<Enc>(storage, n, (cudaStream_t)stream, x_dev, out_dev, n);
}

lbm_status lbm_codec_decode(int storage, const uint16_t* c_dev, float* out_dev, int64_t n, void* stream) {
    if (n > 0 && (!c_dev || !out_dev)) return LBM_ERR_ARG;
    return dispatch<Dec>(storage, n, (cudaStream_t)stream, c_dev, out_dev, n);
}

lbm_status lbm_codec_encode_bits(int storage, uint32_t first, int64_t n, uint16_t* out_dev, void* stream) {
    if (n > 0 && !out_dev) return LBM_ERR_ARG;
    if (n > (int64_t)1 << 32) return LBM_ERR_ARG;
    return dispatch<EncBits>(storage, n, (cudaStream_t)stream, first, out_dev, n);
}

lbm_status lbm_codec_encode_bits_table(int storage, uint32_t first, int64_t n, uint16_t* out_dev, void* stream) {
    if (storage < LBM_P16_0S || storage > LBM_P16_1) return LBM_ERR_UNSUPPORTED;
    if (n > 0 && !out_dev) return LBM_ERR_ARG;
    if (n > (int64_t)1 << 32) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
    const unsigned g = grid_for(n);
    switch (storage) {
    case LBM_P16_0S: EncBitsTable<LBM_P16_0S>::run(g, (cudaStream_t)stream, first, out_dev, n); break;
    case LBM_P16_1S: EncBitsTable<LBM_P16_1S>::run(g, (cudaStream_t)stream, first, out_dev, n); break;
    case LBM_P16_2C: EncBitsTable<LBM_P16_2C>::run(g, (cudaStream_t)stream, first, out_dev, n); break;
    case LBM_P16_0: EncBitsTable<LBM_P16_0>::run(g, (cudaStream_t)stream, first, out_dev, n); break;
    default: EncBitsTable<LBM_P16_1>::run(g, (cudaStream_t)stream, first, out_dev, n); break;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // extern "C"
