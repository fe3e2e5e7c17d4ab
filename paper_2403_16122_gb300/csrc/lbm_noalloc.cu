// lbm_noalloc.cu -- lbm_step_noalloc: one time step of one lattice without a
// handle and without any device allocation. The observable partials of the
// step live in a fixed array that is part of the library's device image.
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// Per-tile observable partials of lbm_step_noalloc (720 KiB per device).
static __device__ __align__(256) double g_noalloc_partials[LBM_NOALLOC_MAX_TILES * lbmk::kObs];

std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the
// array's name only stands for the symbol, so the address is looked up once
// per device (with that device current) and cached.
int scratch_address(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr)
            return LBM_ECUDA;
        g_scratch[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch[dev];
    return LBM_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// [a, a + na) and [b, b + nb) (bytes) share at least one byte.
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" int lbm_step_noalloc(const lbm_params* p, const float* pops_in, const float* aux_in,
                                float* pops_out, float* aux_out, int32_t pitch, double* d_obs,
                                void* cuda_stream) {
    if (!p || !pops_in || !aux_in || !pops_out || !aux_out || !d_obs) return LBM_EINVAL;
    if (!lbmk::params_valid(*p) || pitch < p->nx || pitch % 32 != 0) return LBM_EINVAL;
    if (!aligned16(pops_in) || !aligned16(aux_in) || !aligned16(pops_out) || !aligned16(aux_out))
        return LBM_EINVAL;
    if ((long long)pitch * p->ny * 27 >= (1LL << 31)) return LBM_EINVAL;
    const int tiles_x = (p->nx + 31) / 32;
    const long long n_tiles = (long long)tiles_x * ((p->ny + 7) / 8);
    if (n_tiles > LBM_NOALLOC_MAX_TILES) return LBM_ETOOLARGE;
    // the step reads neighbouring sites of the input while other CTAs write
    // the output: an output buffer may share no byte with any other buffer
    const size_t plane = (size_t)pitch * (size_t)p->ny;
    const size_t pop_b = plane * lbmk::kPopElems * sizeof(float);
    const size_t aux_b = plane * (lbmk::kAuxBlock / 32) * sizeof(float);
    if (overlap(pops_out, pop_b, pops_in, pop_b) || overlap(pops_out, pop_b, aux_in, aux_b) ||
        overlap(pops_out, pop_b, aux_out, aux_b) || overlap(aux_out, aux_b, pops_in, pop_b) ||
        overlap(aux_out, aux_b, aux_in, aux_b))
        return LBM_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != LBM_OK) return rc;
    lbmk::Inst I;
    double L = 0.0;
    lbmk::inst_from_params(*p, &I, &L);
    I.pitch = pitch;
    I.plane = (long long)pitch * p->ny;
    I.pop[0] = const_cast<float*>(pops_in);
    I.pop[1] = pops_out;
    I.aux[0] = const_cast<float*>(aux_in);
    I.aux[1] = aux_out;
    I.part_begin = 0;
    I.part_end = (int)n_tiles;
    I.part_stride = (int)n_tiles;
    cudaError_t e = lbmk::launch_step_noalloc(I, tiles_x, (int)n_tiles, scratch, d_obs,
                                              static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
