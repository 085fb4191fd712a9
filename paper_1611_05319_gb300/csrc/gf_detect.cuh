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
    uint2 *masks;         // [H][NWF] per 32-pixel word of a row: hole bits, not-known bits (bit = column)
    uint8_t *hole_t;      // [NBY][NBX] 1 when the tile holds a hole pixel (cleared before the pack kernel)
    uint8_t *slow_t;      // [NBY][NBX] 1 when a hole pixel may lie within cap of the tile: its distances
                          // are computed; elsewhere every distance is cap + 1
    uint8_t *act_t;       // [NBY][NBX] 1 when the tile holds an annulus pixel (cleared before the
                          // distance kernel): only these tiles' edge, accm and cand entries are written
    uchar2 *dist;         // [H][W] x: Chebyshev distance to the hole, capped at cap + 1; y: 1 on the ring
                          // (distance dR to the hole and no pixel that is not known nearer)
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
    int32_t NWF;          // mask words per row, ceil(W / 32)
};

struct DetectArgs {
    const DetectFrameDev *frames;
    const int32_t *tile_offset;  // [n + 1] first global tile of each frame
    int32_t *active_list;        // [total_tiles] global indices of the tiles holding an annulus pixel
    int32_t *active_count;       // [1] zeroed before the distance kernel
    int32_t *slow_list;          // [total_tiles] global indices of the tiles whose distances are computed
    int32_t *slow_count;         // [1] zeroed before the classify kernel
    const int32_t *word_offset;  // [n + 1] first global mask word of each frame
    int32_t n_frames, total_tiles;
    int32_t rS, rR, dR, annulus, cap;
    float th2, tl2, length, Lambda;
    float wS[2 * DET_MAX_RS + 1];  // normalised taps of g_sigma
    float wR[2 * DET_MAX_RR + 1];  // normalised taps of g_rho
};

struct DetectChunk {
    DetectFrameDev *dst_frames;
    int32_t *dst_to, *dst_wo;
    int32_t first, count, last_chunk, pad;
    DetectFrameDev frames[DET_CHUNK];
    int32_t to[DET_CHUNK + 1];
    int32_t wo[DET_CHUNK + 1];
};

// floats of the tensor kernel's input plane: the window [LI][PI] plus the reach
// of the last run of row outputs
__host__ __device__ inline int detect_plane_floats(int LI, int PI) { return LI * PI + 8; }

// dynamic shared memory of the tensor kernel for radii rS, rR (bytes): the three
// u_sigma planes, then either one channel's input plane and its row-blurred
// plane (odd pitches; 7 rows of padding for the last run of column outputs) or,
// after the blurs, T and m2 on the tile +- 1
inline size_t detect_tensor_smem(int rS, int rR)
{
    const int Rh = rS + rR + 1;
    const int LI = DT + 2 * Rh, LU = DT + 2 * (rR + 1);
    const size_t PI = (size_t)(LI | 1), PQ = (size_t)(LU | 1);
    const size_t blur = (size_t)detect_plane_floats(LI, (int)PI) + (LI + 7) * PQ;
    const size_t tm = 4 * (size_t)(DT + 2) * (DT + 2);
    return 4 * (3 * (size_t)LU * LU + (blur > tm ? blur : tm));
}

// mask words per row of the distance kernel's window (tile +- cap, widened to
// whole 32-pixel words)
__host__ __device__ inline int detect_window_words(int cap) { return 1 + 2 * ((cap + 31) / 32); }

// dynamic shared memory of the distance kernel for the cap (bytes): the window's
// hole and not-known masks with a zero rim of one word and one row, double-
// buffered for the dilation, and the not-known masks as loaded
inline size_t detect_dist_smem(int cap)
{
    const size_t L = DT + 2 * (size_t)cap, NW = (size_t)detect_window_words(cap);
    return 4 * 5 * (L + 2) * (NW + 2);
}

__global__ void upload_detect_kernel(const __grid_constant__ DetectChunk c);
__global__ void detect_pack_kernel(const __grid_constant__ DetectArgs a, int total_words);
__global__ void detect_classify_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_dist_kernel(const __grid_constant__ DetectArgs a);
__global__ void detect_dist_warp_kernel(const __grid_constant__ DetectArgs a);  // cap <= 31
constexpr int DET_WARP_DIST_MAX_CAP = 31;
template <int RS>
__global__ void detect_tensor_kernel(const __grid_constant__ DetectArgs a);
// the instantiation for radius rS (1..DET_MAX_RS), and its launch
const void *detect_tensor_entry(int rS);
cudaError_t launch_detect_tensor(int rS, unsigned grid, size_t smem, cudaStream_t st, const DetectArgs &a);
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
