// Particle-filter kernels (Section 2.2, Section 3.3 DA steps (I)-(V),
// perturbation of Section 4.4), all on the device so the ensemble never
// leaves HBM: gauge sampling, weights / N_eff / systematic resampling /
// slot assignment in one single-block kernel, and a grid-stride copy of the
// duplicated members' states.  Also the per-member storage and max-depth
// reductions.
#include "flood_internal.cuh"
#include "pf_kernels.cuh"

namespace flood {

namespace {

// DA step (I): y[i][k] = depth of member i at gauge cell k.
__global__ void gauge_kernel(const float* __restrict__ state, const MemberClock* __restrict__ ms,
                             const int32_t* __restrict__ cells, int G, int M, int ld, int nx,
                             size_t plane, float* __restrict__ y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * G) return;
    const int m = t / G, k = t % G;
    const int cell = cells[k];
    const int r = cell / nx, c = cell % nx;
    const float* h = state + (size_t)(ms[m].cur * M + m) * 3 * plane;
    y[t] = h[(size_t)r * ld + c];
}

// DA steps (II)-(IV) and the bookkeeping of step (V), one block.
// Sums run sequentially in index order on one thread (FP64), so the
// cumulative weights are formed exactly as the sequential definition.
__global__ void pf_kernel(PfArgs a)
{
    extern __shared__ double sm[];
    double* lw = sm;                       // [M] log-weights, then weights
    float* rm_old = (float*)(sm + a.M);    // [M]
    float* sc_old = rm_old + a.M;          // [M]
    const int M = a.M, G = a.G;

    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double chi2 = 0.0;
        for (int k = 0; k < G; ++k) {
            double s = a.sigma_rel > 0.0 ? a.sigma_rel * a.d[k] : a.sigma[k];
            double e = ((double)a.y[(size_t)i * G + k] - a.d[k]) / s;
            chi2 += e * e;
        }
        lw[i] = log(a.w[i]) - 0.5 * chi2;   // log of Eq. 10
        rm_old[i] = a.rain_mult[i];
        sc_old[i] = a.scale[i];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;

    double lmax = -INFINITY;
    for (int i = 0; i < M; ++i) lmax = lw[i] > lmax ? lw[i] : lmax;
    if (!(lmax > -INFINITY)) {  // every weight zero: leave the ensemble untouched
        *a.status = 1;
        *a.resampled = 0;
        *a.n_copy = 0;
        *a.neff = 0.0;
        for (int i = 0; i < M; ++i) a.idx[i] = i;
        return;
    }
    double sum = 0.0;
    for (int i = 0; i < M; ++i) sum += exp(lw[i] - lmax);
    double s2 = 0.0;
    for (int i = 0; i < M; ++i) {
        double w = exp(lw[i] - lmax) / sum;  // Eq. 11
        lw[i] = w;
        a.w_post[i] = w;
        s2 += w * w;
    }
    const double neff = 1.0 / s2;           // Eq. 12
    *a.neff = neff;
    *a.status = 0;
    const bool resample = a.force || neff < a.n_thr_frac * (double)M;
    *a.resampled = resample ? 1 : 0;
    if (!resample) {
        for (int i = 0; i < M; ++i) {
            a.w[i] = lw[i];
            a.idx[i] = i;
        }
        *a.n_copy = 0;
        return;
    }
    // systematic resampling: particle i owns [c_{i-1}, c_i)
    int32_t* idx = a.idx;
    double acc = 0.0;
    int i = 0;
    double ci = 0.0;
    // running cumulative sum, c_{M-1} forced to 1
    acc = lw[0];
    ci = (M == 1) ? 1.0 : acc;
    for (int j = 0; j < M; ++j) {
        const double uj = (a.u + (double)j) / (double)M;
        while (i < M - 1 && ci <= uj) {
            ++i;
            acc += lw[i];
            ci = (i == M - 1) ? 1.0 : acc;
        }
        idx[j] = i;
    }
    // DA step (V): duplicates per particle; survivors keep their slot, extra
    // copies (in particle order) fill dropped slots (in slot order)
    int32_t* cnt = a.cnt;
    for (int p = 0; p < M; ++p) cnt[p] = 0;
    for (int j = 0; j < M; ++j) cnt[idx[j]]++;
    int next = 0, nc = 0;
    for (int s = 0; s < M; ++s) {
        int src;
        if (cnt[s] >= 1) {
            src = s;
        } else {
            while (cnt[next] <= 1) ++next;
            src = next;
            cnt[next]--;
            a.copy_dst[nc] = s;
            a.copy_src[nc] = src;
            ++nc;
        }
        a.src[s] = src;
    }
    *a.n_copy = nc;
    // parameters follow their particle; rain multiplier perturbed by beta
    for (int s = 0; s < M; ++s) {
        a.rain_mult[s] = rm_old[a.src[s]] * a.beta[s];
        a.scale[s] = sc_old[a.src[s]];
        a.w[s] = 1.0 / (double)M;
    }
    // the copied members inherit their source's maximum depth (same time)
    for (int q = 0; q < nc; ++q) a.ms[a.copy_dst[q]].hmax_bits = a.ms[a.copy_src[q]].hmax_bits;
}

// DA step (V): copy the duplicated particles' h, qx, qy planes into the
// dropped slots.  Grid-stride over (copy, plane, float4); reads the device
// copy count so that the launch needs no host synchronisation.
__global__ void copy_kernel(float* __restrict__ state, const MemberClock* __restrict__ ms,
                            const int32_t* __restrict__ n_copy, const int32_t* __restrict__ dsts,
                            const int32_t* __restrict__ srcs, int M, size_t plane4)
{
    const int nc = *n_copy;
    if (nc == 0) return;
    const size_t per = 3 * plane4;  // float4s per member
    const size_t total = (size_t)nc * per;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / per);
        const size_t e = t - (size_t)q * per;
        const int d = dsts[q], s = srcs[q];
        const float4* from = reinterpret_cast<const float4*>(state) + (size_t)(ms[s].cur * M + s) * per;
        float4* to = reinterpret_cast<float4*>(state) + (size_t)(ms[d].cur * M + d) * per;
        to[e] = from[e];
    }
}

// Systematic resampling alone (DA step (IV)), one thread.
__global__ void resample_kernel(int M, const double* __restrict__ w, double u,
                                int32_t* __restrict__ idx)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = w[0];
    double ci = (M == 1) ? 1.0 : acc;
    int i = 0;
    for (int j = 0; j < M; ++j) {
        const double uj = (u + (double)j) / (double)M;
        while (i < M - 1 && ci <= uj) {
            ++i;
            acc += w[i];
            ci = (i == M - 1) ? 1.0 : acc;
        }
        idx[j] = i;
    }
}

// Per-member FP64 storage partials: block b of member m sums a fixed set of
// rows in a fixed order; the final pass adds the partials in index order.
__global__ void storage_partial_kernel(const float* __restrict__ state,
                                       const MemberClock* __restrict__ ms, int M, int ny, int nx,
                                       int ld, size_t plane, int rows_per_block,
                                       double* __restrict__ part)
{
    const int m = blockIdx.y;
    const float* h = state + (size_t)(ms[m].cur * M + m) * 3 * plane;
    const int r0 = blockIdx.x * rows_per_block, r1 = min(r0 + rows_per_block, ny);
    double acc = 0.0;
    for (int r = r0; r < r1; ++r)
        for (int c = threadIdx.x; c < nx; c += blockDim.x) acc += (double)h[(size_t)r * ld + c];
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)m * gridDim.x + blockIdx.x] = red[0];
}

__global__ void storage_final_kernel(const double* __restrict__ part, int nb, int M,
                                     double area, double* __restrict__ out)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)m * nb + b];
    out[m] = acc * area;
}

// Maximum depth of each member's current state (initialisation of the
// Eq. 4 input); non-negative floats order like their bit patterns.
__global__ void hmax_kernel(const float* __restrict__ state, MemberClock* __restrict__ ms, int M,
                            int ny, int nx, int ld, size_t plane)
{
    const int m = blockIdx.y;
    const float* h = state + (size_t)(ms[m].cur * M + m) * 3 * plane;
    unsigned best = 0u;
    const size_t n = (size_t)ny * nx;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / nx, c = t % nx;
        best = max(best, __float_as_uint(fmaxf(h[r * ld + c], 0.0f)) & 0x7fffffffu);
    }
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0) atomicMax(&ms[m].hmax_bits, best);
}

}  // namespace

void launch_gauge(const float* state, const MemberClock* ms, const int32_t* cells, int G, int M,
                  int ld, int nx, size_t plane, float* y, cudaStream_t s)
{
    const int n = M * G;
    gauge_kernel<<<(n + 127) / 128, 128, 0, s>>>(state, ms, cells, G, M, ld, nx, plane, y);
}

void launch_pf(const PfArgs& a, cudaStream_t s)
{
    const size_t shm = sizeof(double) * a.M + 2 * sizeof(float) * a.M;
    pf_kernel<<<1, 128, shm, s>>>(a);
}

void launch_copy(float* state, const MemberClock* ms, const int32_t* n_copy, const int32_t* dsts,
                 const int32_t* srcs, int M, size_t plane, int n_sm, cudaStream_t s)
{
    copy_kernel<<<n_sm * 4, 512, 0, s>>>(state, ms, n_copy, dsts, srcs, M, plane / 4);
}

void launch_resample(int M, const double* w, double u, int32_t* idx, cudaStream_t s)
{
    resample_kernel<<<1, 32, 0, s>>>(M, w, u, idx);
}

int launch_storage(const float* state, const MemberClock* ms, int M, int ny, int nx, int ld,
                   size_t plane, double area, double* part, int part_cap, double* out,
                   cudaStream_t s)
{
    const int rows = 16;
    const int nb = (ny + rows - 1) / rows;
    if (nb > part_cap) return -1;
    storage_partial_kernel<<<dim3(nb, M), 256, 0, s>>>(state, ms, M, ny, nx, ld, plane, rows, part);
    storage_final_kernel<<<(M + 127) / 128, 128, 0, s>>>(part, nb, M, area, out);
    return 0;
}

void launch_hmax(const float* state, MemberClock* ms, int M, int ny, int nx, int ld, size_t plane,
                 int n_sm, cudaStream_t s)
{
    const size_t n = (size_t)ny * nx;
    int bx = (int)((n + 255) / 256);
    if (bx > n_sm * 2) bx = n_sm * 2;
    hmax_kernel<<<dim3(bx, M), 256, 0, s>>>(state, ms, M, ny, nx, ld, plane);
}

}  // namespace flood
