// Host-side inputs of the in-place host-buffer fill (gf_fill_batched_host with
// out_rgba == rgba on device-accessible host memory) that the fill kernel does
// not read itself: a caller-given guide field is needed at hole pixels only, so
// only the guide of the 8x8 tiles holding a hole pixel is read from the caller's
// buffer (the fill kernel gathers the colours it needs, near the holes, and
// writes the hole pixels' colours and the shell map back).
//
// Kernels (up to HOSTIO_MAX frames per launch; one frame per blockIdx.y, except the
// gather, a small persistent grid over the launch's frames):
//   hostio_holes_kernel    per 8x8 tile: does it hold a hole pixel (labels, read
//                          from the caller's buffer where host_labels is set)
//   hostio_gather_kernel   host -> device colours of the tiles next to a hole tile
//                          (where host_rgba is set) and guide of the hole tiles
//                          (where host_guide is set)
//   hostio_write_back_kernel   after the fill: the hole pixels' colours (and
//                          shell values) into the caller's buffers
// The gather runs one warp per strip of 8 rows x 256 columns, lane l on the
// columns l, l + 32, ... so that every access of a warp covers contiguous bytes
// of a row.  Every kernel issues a batch of loads before the stores that use them:
// a store may alias a later load, so the compiler keeps program order, and
// alternating loads and stores would leave one host round trip in flight per warp.

#include "gf_internal.cuh"

namespace gf {

namespace {
constexpr unsigned FULLM = 0xffffffffu;
}

// The strip of warp `unit`: tile row ty, columns of tiles 32 s .. 32 s + 31.
// Returns false (for the whole warp) past the frame's last strip.
__device__ __forceinline__ bool hostio_strip(const HostIOFrame &F, int &ty, int &s)
{
    const int strips = (F.TW + 31) >> 5;
    const int unit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (unit >= F.TH * strips) return false;
    ty = unit / strips;
    s = unit - ty * strips;
    return true;
}

// Per 8x8 tile: does it hold a hole pixel.  With host_labels set, the labels are
// read from the caller's host buffer and written to the device copy on the way.
// One warp per strip of 8 rows x 32 tiles, lane l on tile column 32 s + l.
__global__ void __launch_bounds__(256) hostio_holes_kernel(const __grid_constant__ HostIOArgs a)
{
    if ((int)blockIdx.y >= a.n) return;
    const HostIOFrame &F = a.f[blockIdx.y];
    int ty, s;
    if (!hostio_strip(F, ty, s)) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const int tx = s * 32 + lane;
    if (tx >= F.TW) return;
    const int x0 = tx * TILE;
    const uint8_t *src = F.host_labels ? F.host_labels : F.labels;
    const bool vec = (F.W & 7) == 0 && (reinterpret_cast<uintptr_t>(src) & 7u) == 0 &&
                     (reinterpret_cast<uintptr_t>(F.labels) & 7u) == 0;
    bool any = false;
    if (vec) {
        // the tile's 8 rows in flight together
        uint2 v[TILE];
#pragma unroll
        for (int r = 0; r < TILE; r++) {
            const int y = ty * TILE + r;
            v[r] = y < F.H ? *reinterpret_cast<const uint2 *>(src + (size_t)y * F.W + x0) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int r = 0; r < TILE; r++) {
            const int y = ty * TILE + r;
            if (y >= F.H) break;
            if (F.host_labels) *reinterpret_cast<uint2 *>(F.labels + (size_t)y * F.W + x0) = v[r];
#pragma unroll
            for (int c = 0; c < 8; c++) any |= (((c < 4 ? v[r].x : v[r].y) >> (8 * (c & 3))) & 0xffu) == 1u;
        }
    } else {
        for (int r = 0; r < TILE; r++) {
            const int y = ty * TILE + r;
            if (y >= F.H) break;
            const size_t o = (size_t)y * F.W + x0;
            for (int c = 0; c < TILE && x0 + c < F.W; c++) {
                const uint8_t l = src[o + c];
                if (F.host_labels) F.labels[o + c] = l;
                any |= l == 1;
            }
        }
    }
    F.tile_hole[ty * F.TW + tx] = any ? 1 : 0;
}

// A small persistent grid (a third of the SMs; the host link needs only a few
// hundred KB in flight) that leaves the other SMs to the guide-field kernel running beside
// it: every warp walks the launch's frames in order and takes every nw-th strip.
__device__ __forceinline__ void hostio_gather_strip(const HostIOFrame &F, int ty, int s)
{
    const int lane = threadIdx.x & 31;
    const int tx = s * 32 + lane;
    // lane l: is tile 32 s + l next to (or holding) a hole pixel; does it hold one
    bool rel = false, own = false;
    if (tx < F.TW) {
        own = F.tile_hole[ty * F.TW + tx] != 0;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int nx = tx + dx, ny = ty + dy;
                if (nx >= 0 && ny >= 0 && nx < F.TW && ny < F.TH && F.tile_hole[ny * F.TW + nx]) rel = true;
            }
    }
    const unsigned relm = __ballot_sync(FULLM, rel), ownm = __ballot_sync(FULLM, own);
    if (!relm) return;
    const int xs = s * 32 * TILE;
    // two rows (16 colours a lane) in flight at a time
    for (int r0 = 0; r0 < TILE; r0 += 2) {
        float4 c[16];
        float2 g[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int y = ty * TILE + r0 + (k >> 3), p = lane + 32 * (k & 7), x = xs + p;
            const size_t o = (size_t)y * F.W + x;
            const bool in = y < F.H && x < F.W;
            c[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            g[k] = make_float2(0.f, 0.f);
            if (F.host_rgba && in && ((relm >> (p >> 3)) & 1u)) c[k] = F.host_rgba[o];
            if (F.host_guide && in && ((ownm >> (p >> 3)) & 1u)) g[k] = F.host_guide[o];
        }
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int y = ty * TILE + r0 + (k >> 3), p = lane + 32 * (k & 7), x = xs + p;
            const size_t o = (size_t)y * F.W + x;
            const bool in = y < F.H && x < F.W;
            if (F.host_rgba && in && ((relm >> (p >> 3)) & 1u)) F.dev_rgba[o] = c[k];
            if (F.host_guide && in && ((ownm >> (p >> 3)) & 1u)) F.dev_guide[o] = g[k];
        }
    }
}

__global__ void __launch_bounds__(256) hostio_gather_kernel(const __grid_constant__ HostIOArgs a)
{
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int fi = 0; fi < a.n; fi++) {
        const HostIOFrame &F = a.f[fi];
        const int strips = (F.TW + 31) >> 5;
        for (int u = gw; u < F.TH * strips; u += nw) hostio_gather_strip(F, u / strips, u - (u / strips) * strips);
    }
}

// After the fill: the colours of the hole pixels into the caller's host image
// and, where host_shell is set, their shell values into the caller's host shell
// map (which a bulk copy taken while the fill ran filled with every other entry,
// final since the init pass).  One warp per strip of 8 rows x 256 columns.
__global__ void __launch_bounds__(256) hostio_write_back_kernel(const __grid_constant__ HostIOArgs a)
{
    if ((int)blockIdx.y >= a.n) return;
    const HostIOFrame &F = a.f[blockIdx.y];
    int ty, s;
    if (!hostio_strip(F, ty, s)) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const int tx = s * 32 + lane;
    const bool own = tx < F.TW && F.tile_hole[ty * F.TW + tx] != 0;
    const unsigned ownm = __ballot_sync(FULLM, own);
    if (!ownm) return;
    const int xs = s * 32 * TILE;
    for (int r = 0; r < TILE; r++) {
        const int y = ty * TILE + r;
        if (y >= F.H) break;
        const size_t row = (size_t)y * F.W;
        // the row's labels, then its hole colours and shell values, all loaded before
        // the host stores
        bool h[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int p = lane + 32 * i, x = xs + p;
            h[i] = x < F.W && ((ownm >> (p >> 3)) & 1u) && F.labels[row + x] == 1;
        }
        float4 c[8];
        int32_t sh[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const size_t o = row + xs + lane + 32 * i;
            c[i] = h[i] ? F.dev_rgba[o] : make_float4(0.f, 0.f, 0.f, 0.f);
            sh[i] = (h[i] && F.host_shell) ? F.dev_shell[o] : 0;
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const size_t o = row + xs + lane + 32 * i;
            if (h[i]) {
                F.host_rgba[o] = c[i];
                if (F.host_shell) F.host_shell[o] = sh[i];
            }
        }
    }
}

}  // namespace gf
