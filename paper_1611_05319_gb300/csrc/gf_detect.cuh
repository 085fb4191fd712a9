// Automatic spline detection (Section 3.3): device-side declarations.
#pragma once

#include "gf_internal.cuh"

namespace gf {

constexpr int DT = 32;            // detection tile side (pixels)
constexpr int DET_THREADS = 256;  // 8 warps; warp w takes tile rows w, w + 8, w + 16, w + 24
constexpr int DET_MAX_RS = 8;     // radius ceil(2 sigma) of g_sigma, sigma <= 4
constexpr int DET_MAX_RR = 16;    // radius ceil(2 rho) of g_rho, rho <= 8
constexpr int DET_MAX_CAP = 97;   // distance cap dR + annulus + 1
constexpr int DET_CHUNK = 64;     // frame descriptors per upload kernel
constexpr int DET_SCAN_THREADS = 1024;

struct DetectFrameDev {
    int32_t H, W, NBX, NBY;
    const float4 *rgba;
    const uint8_t *labels;
    uchar2 *dist;         // [H][W] Chebyshev distance to the hole / to any pixel not known, capped at cap + 1
    uint8_t *active;      // [NBY][NBX] 1 when the tile holds an annulus pixel
    uint8_t *edge;        // [H][W] after suppression and thresholds: 0, 1 weak, 2 strong (annulus only)
    int32_t *parent;      // [H][W] union-find forest over edge pixels
    int32_t *mark;        // [H][W] set at roots whose component holds a strong pixel
    float4 *cand;         // [H][W] at ring pixels on an edge: spline end x, end y, weight
    uint32_t *accm;       // [H][NBX] accepted ring pixels of each 32-pixel row segment (bit = column)
    uint32_t *accpos;     // [H][NBX] output position of the segment's first accepted pixel
    float2 *pts;          // [max_splines][2]
    float *weight;        // [max_splines]
    int32_t *offsets;     // [max_splines + 1]
    int32_t *base;        // [max_splines] or null
    uint8_t *edges_out;   // [H][W] or null
    int32_t *result;      // [2]
    int32_t max_splines;
    int32_t pad;
};

struct DetectArgs {
    const DetectFrameDev *frames;
    const int32_t *tile_offset;  // [n + 1] first global tile of each frame
    int32_t n_frames, total_tiles;
    int32_t rS, rR, dR, annulus, cap;
    float th2, tl2, length, Lambda;
    float wS[2 * DET_MAX_RS + 1];  // normalised taps of g_sigma
    float wR[2 * DET_MAX_RR + 1];  // normalised taps of g_rho
};

struct DetectChunk {
    DetectFrameDev *dst_frames;
    int32_t *dst_to;
    int32_t first, count, last_chunk, pad;
    DetectFrameDev frames[DET_CHUNK];
    int32_t to[DET_CHUNK + 1];
};

// shared memory of the tensor kernel for radii rS, rR (bytes)
inline size_t detect_tensor_smem(int rS, int rR)
{
    const size_t Rh = (size_t)rS + rR + 1;
    const size_t LI = DT + 2 * Rh, LU = DT + 2 * ((size_t)rR + 1), LT = DT + 2 * (size_t)rR;
    const size_t A = 3 * LI * LI;
    const size_t B = 3 * LI * LU > 3 * LT * LT ? 3 * LI * LU : 3 * LT * LT;
    return 4 * (A + B + (size_t)(DT + 2) * (DT + 2));
}

// shared memory of the distance kernel for the cap (bytes)
inline size_t detect_dist_smem(int cap)
{
    const size_t L = DT + 2 * (size_t)cap;
    return L * L + 2 * L * DT;
}

__global__ void upload_detect_kernel(const __grid_constant__ DetectChunk c);
__global__ void detect_dist_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_tensor_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_union_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_mark_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_accept_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_scan_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_write_kernel(const __grid_constant__ DetectArgs a);

// per-spline weights of a guide-field request: frames [first, first + count)
struct WeightChunk {
    const float *w[DESC_CHUNK];
    int32_t first, count;
};
__global__ void spline_weight_kernel(const __grid_constant__ GuideArgs a, const __grid_constant__ WeightChunk c);

}  // namespace gf
