// K5: USPG -> Cartesian resampling for display (Sec. II.B).
//
// POINT mode: one thread per pixel of the plane (all slabs share the
// classification); the pixel centre is classified
// into (ring, sector) with the same FP64 rule as the coefficient midpoints
// (ring = floor(rho / r), sector = floor((atan2 + 1e-12) n_g / 2 pi)), so a
// pixel centre on a radial boundary belongs to the sector that starts there.
// BIJECTION mode (4(2n-1) grids): square ring n of a 2N x 2N image has as many
// pixels as polar ring n has cells (Sec. II.A); the pixels are numbered
// counter-clockwise from the +x axis along the square's perimeter (walk
// index from integer pixel coordinates, no trigonometry) and pixel j of
// square ring n shows cell H_n + j.
#include "internal.cuh"

namespace uspg {

// One thread per pixel of the nx x ny plane: the cell under the pixel centre
// is the same in every slab, so it is classified once and the slabs are
// copied in a loop (consecutive threads write consecutive pixels).
__global__ void k_resample_point(const float *__restrict__ f, const RingEntry *__restrict__ rt, int n_rings, double r,
                                 long long cps, int n_slabs, int nx, int ny, float *__restrict__ out)
{
    long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)nx * ny;
    if (pix >= per) return;
    int b = (int)(pix / nx), a = (int)(pix % nx);
    double R = (double)n_rings * r;
    double x = -R + ((double)a + 0.5) * (2.0 * R / (double)nx);
    double y = -R + ((double)b + 0.5) * (2.0 * R / (double)ny);
    double rho = sqrt(x * x + y * y);
    long long cell = -1;
    if (rho < R) {
        long long ring = (long long)floor(rho / r);
        if (ring > n_rings - 1) ring = n_rings - 1;
        int ng = rt[ring].ng;
        double phi = atan2(y, x);
        if (phi < 0.0) phi += kTwoPi;
        long long sec = (long long)floor(((phi + kNudge) * (double)ng) / kTwoPi);
        if (sec >= ng) sec -= ng;
        cell = rt[ring].head + sec;
    }
    for (int slab = 0; slab < n_slabs; slab++)
        out[slab * per + pix] = cell >= 0 ? f[(long long)slab * cps + cell] : 0.0f;
}

// Position of pixel (a, b) of a 2N x 2N image along its square ring.
__device__ __forceinline__ void square_ring_index(int a, int b, int N, int *ring1, int *j)
{
    // doubled coordinates are odd integers: X = 2a - 2N + 1, Y = 2b - 2N + 1
    int X = 2 * a - 2 * N + 1, Y = 2 * b - 2 * N + 1;
    int ax = X < 0 ? -X : X, ay = Y < 0 ? -Y : Y;
    int M = ax > ay ? ax : ay;  // = 2n - 1
    int n = (M + 1) / 2;
    int idx;
    if (X == M && Y > 0) idx = (Y - 1) / 2;                  // right edge, upper half
    else if (Y == M) idx = (n - 1) + (M - X) / 2;           // top edge, right to left
    else if (X == -M) idx = (3 * n - 2) + (M - Y) / 2;      // left edge, top to bottom
    else if (Y == -M) idx = (5 * n - 3) + (X + M) / 2;      // bottom edge, left to right
    else idx = (7 * n - 4) + (Y + M) / 2;                   // right edge, lower half
    *ring1 = n;
    *j = idx;
}

__global__ void k_resample_bijection(const float *__restrict__ f, const RingEntry *__restrict__ rt, int N,
                                     long long cps, int n_slabs, float *__restrict__ out)
{
    long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int W = 2 * N;
    long long per = (long long)W * W;
    if (pix >= per) return;
    int b = (int)(pix / W), a = (int)(pix % W);
    int n, j;
    square_ring_index(a, b, N, &n, &j);
    long long cell = rt[n - 1].head + j;
    for (int slab = 0; slab < n_slabs; slab++) out[slab * per + pix] = f[(long long)slab * cps + cell];
}

uspg_status launch_resample(uspg_ctx *c, int mode, int nx, int ny, float *out, cudaStream_t s)
{
    int ns = c->scan.geometry == USPG_CONE_3D ? c->n_slabs : 1;
    const int TB = 256;
    const float *f = c->d_f;
    if (c->mir.on) {  // mirrored image pairs -> standard layout (a buffer the context keeps)
        if (!c->d_rs_std) USPG_CUDA(c, cudaMalloc(&c->d_rs_std, sizeof(float) * c->n_cells));
        USPG_CUDA(c, image_from_pairs(c, c->d_f, c->d_rs_std, s));
        f = c->d_rs_std;
    }
    if (mode == USPG_RESAMPLE_POINT) {
        long long n = (long long)nx * ny;
        k_resample_point<<<(unsigned)((n + TB - 1) / TB), TB, 0, s>>>(f, c->d_ring, c->n_rings, c->r,
                                                                      c->cells_per_slab, ns, nx, ny, out);
    } else {
        long long n = 4LL * c->n_rings * c->n_rings;
        k_resample_bijection<<<(unsigned)((n + TB - 1) / TB), TB, 0, s>>>(f, c->d_ring, c->n_rings,
                                                                          c->cells_per_slab, ns, out);
    }
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

}  // namespace uspg
