// TMA-staged reverse stencil (same arithmetic and results, bit for bit, as
// adjoint_kernel.cu, through the shared row code of adjoint_row.cuh).
//
// The direct-load adjoint kernel needs about 120 registers per thread, so
// only four CTAs of four warps fit on an SM and its loads cannot keep enough
// bytes in flight: it ran at about a third of the HBM bandwidth.  Here each
// warp streams its rows through a ring of shared-memory stages filled by the
// tensor memory accelerator, one row of all ten planes it reads per stage:
// the state before the step (h, qx, qy), the depth after it, the
// sensitivities lambda (h, qx, qy), the bed and roughness (with land cover
// the bed and the class codes), and the member's Manning gradient, each 136
// columns wide (the warp's 128 plus a 4-column halo on each side).  Lane 0 keeps kNS - 1 rows in flight ahead of the row
// being computed.  Every mbarrier wait is bounded: on timeout the kernel
// records FLOOD_ERR_TIMEOUT, waits (bounded) for its own copies in flight,
// and returns.
#include "adjoint.cuh"
#include "adjoint_row.cuh"
#include "tma.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;
constexpr int kNS = 3;                          // stages per warp
constexpr int kBox = kSpan + 8;                 // columns per tile row
// float offsets inside a stage (each part starts on a 128-byte boundary)
constexpr int kSt = 0;                          // h, qx, qy before the step: 3 x kBox
constexpr int kHa = 416;                        // depth after the step: kBox
constexpr int kLam = 576;                       // lambda h, qx, qy: 3 x kBox
constexpr int kZ = 992;                         // bed: kBox
constexpr int kN = kZ + kBox;                   // roughness: kBox
constexpr int kGn = 1280;                       // Manning gradient: kBox
constexpr int kStageBytes = 5760;
constexpr uint32_t kRowBytes = kBox * 4;
constexpr long long kWaitBudget = 200000000LL;  // clock cycles (~0.1 s) before giving up

static_assert(kHa * 4 >= 3 * kBox * 4 && kHa % 32 == 0, "stage layout");
static_assert(kLam * 4 >= (kHa + kBox) * 4 && kLam % 32 == 0, "stage layout");
static_assert(kZ * 4 >= (kLam + 3 * kBox) * 4 && kZ % 32 == 0, "stage layout");
static_assert(kGn * 4 >= (kN + kBox) * 4 && kGn % 32 == 0, "stage layout");
static_assert(kStageBytes >= (kGn + kBox) * 4 && kStageBytes % 128 == 0, "stage layout");
// Land cover: the roughness plane's place holds each cell's class code (a
// uint32), staged with the bed as in the forward step.

__device__ __forceinline__ void lds4(float (&v)[4], const float* p)
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// LC: land cover: the roughness, runoff share and drainage flag of every
// cell from its class (the codes come with the staged rows, the member's
// class table lives in lanes 0..3 and is read by shuffle, so every lane takes
// part in each lookup, outside lane-dependent branches).
template <int WM, int LIM, bool LC = false>
__global__ void __launch_bounds__(32 * WM, WM == 4 ? 3 : 12) adjoint_tma_kernel(
    const __grid_constant__ AdjTmaArgs t)
{

    extern __shared__ unsigned char smem_raw[];
    const AdjArgs& a = t.a;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int m = blockIdx.x * WM + w;
    const int span = blockIdx.y;
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps; no block-wide barriers below

    const int nx = a.nx, ny = a.ny, ld = a.ld;
    const size_t plane = a.plane, mstride = 3 * plane;
    const int c = c0 + 4 * lane;
    const bool act = c < nx;
    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, ny);
    const float* __restrict__ lin = a.lam + ((size_t)a.lam_in * a.M + m) * mstride;
    float* __restrict__ lout = a.lam + ((size_t)(1 - a.lam_in) * a.M + m) * mstride;

    const int j = a.seg_end[m] - 1 - a.rev_i;
    if (j < a.seg_first) {  // member idle in this launch: carry lambda over
        if (act)
            for (int r = r0; r < r1; ++r)
                for (int q = 0; q < 3; ++q) {
                    const size_t o = q * plane + (size_t)r * ld + c;
                    *reinterpret_cast<float4*>(lout + o) = ldg4(lin + o);
                }
        return;
    }
    if (*reinterpret_cast<volatile const int*>(a.err) & 2) return;  // an earlier wait gave up

    const MemberPlan pl = a.log[(size_t)m * a.dt_log_cap + j];
    FaceK k;
    k.gdt_dx = pl.gdt_dx;
    k.gdt = pl.gdt;
    k.dx_4dt = pl.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = 0.0f;  // no inflow boundary here
    k.in_r0 = k.in_r1 = 0;
    const float T = pl.dt_dx;
    const float s = a.scale[m];
    const float s_half = 0.5f * s;
    const bool interior = c0 + kSpan < nx;  // no east edge in this span
    float* __restrict__ gn = a.gn ? a.gn + (size_t)m * plane : nullptr;

    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    const uint32_t bar0 = smem_u32(base) + 8u * kNS * w;
    unsigned char* my_stages = base + 128 * ((8 * kNS * WM + 127) / 128) + kNS * kStageBytes * w;
    const uint32_t stage0 = smem_u32(my_stages);

    const int slot = j - a.seg_first;                 // seg slot of the state before the step
    const int p_before = (slot * a.M + m) * 3;        // plane index in the seg map
    const int p_after = ((slot + 1) * a.M + m) * 3;   // depth plane after the step
    const int p_lam = (a.lam_in * a.M + m) * 3;
    const uint32_t tx = kRowBytes * (gn ? 10u : 9u);
    const int ra = r0 > 0 ? r0 - 1 : r0;   // first row loaded (north halo)
    const int rb = min(r1 + 1, ny);        // one past the last row loaded

    if (lane == 0) {
        for (int i = 0; i < kNS; ++i) mbar_init(bar0 + 8u * i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    int issued = ra;  // rows [ra, issued) have been requested
    auto issue = [&](int row) {
        const int sidx = (row - ra) % kNS;
        const uint32_t bar = bar0 + 8u * sidx;
        const uint32_t dsts = stage0 + kStageBytes * sidx;
        mbar_arrive_expect_tx(bar, tx);
        tma_load_3d(dsts + 4 * kSt, &t.seg_map, c0 - 4, row, p_before, bar);
        tma_load_3d(dsts + 4 * kHa, &t.seg1_map, c0 - 4, row, p_after, bar);
        tma_load_3d(dsts + 4 * kLam, &t.lam_map, c0 - 4, row, p_lam, bar);
        tma_load_3d(dsts + 4 * kZ, &t.static_map, c0 - 4, row, 0, bar);
        if (gn) tma_load_3d(dsts + 4 * kGn, &t.gn_map, c0 - 4, row, m, bar);
    };
    for (; issued < rb && issued < ra + kNS; ++issued)
        if (lane == 0) issue(issued);
    auto wait_row = [&](int row) -> bool {
        const int kk = row - ra;
        return mbar_wait_bounded(bar0 + 8u * (kk % kNS), (kk / kNS) & 1, kWaitBudget);
    };
    auto row_ptr = [&](int row) -> const float* {
        return reinterpret_cast<const float*>(my_stages + kStageBytes * ((row - ra) % kNS));
    };
    // recycle the oldest stage for the next row in line
    auto release = [&]() {
        __syncwarp();
        if (issued < rb) {
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(issued);
            }
            ++issued;
        }
    };
    int waited = ra;  // rows [ra, waited) have landed
    auto drain_and_fail = [&]() {
        if (lane == 0) atomicOr(a.err, 2);
        for (int row = waited; row < issued; ++row) wait_row(row);  // bounded each
    };

    const int x0 = 4 + 4 * lane;  // this lane's first cell in a tile row
    // land cover: lane q of every group of four holds class q's roughness,
    // runoff share and drainage flag for this member
    float ln = 0.0f, lro = 0.0f, ldr = 0.0f;
    if (LC) {
        const int q = lane & 3;
        ln = a.lc_n[(size_t)m * 4 + q];
        lro = a.lc_runoff[q];
        ldr = a.lc_drains[q];
    }
    // the classes of the lane's four cells in a staged row, one byte each
    auto cls4 = [&](const float* R) -> uint32_t {
        const uint4 q = *reinterpret_cast<const uint4*>(R + kN + x0);
        return __byte_perm(__byte_perm(q.x, q.y, 0x0040u), __byte_perm(q.z, q.w, 0x0040u), 0x5410u);
    };
    // roughness of the lane's four cells / of one cell of a staged row (with
    // land cover by shuffle: every lane calls these; the shuffle reads the
    // five low bits of its source lane, where a class byte sits alone)
    auto n4 = [&](float (&nv)[4], const float* R) {
        if (LC) {
            const uint32_t wc = cls4(R);
#pragma unroll
            for (int q = 0; q < 4; ++q) nv[q] = __shfl_sync(0xffffffffu, ln, (int)(wc >> (8 * q)));
        } else {
            lds4(nv, R + kN + x0);
        }
    };
    auto n1 = [&](const float* R, int x) -> float {
        return LC ? __shfl_sync(0xffffffffu, ln, (int)__float_as_uint(R[kN + x])) : R[kN + x];
    };
    float hC[4], zC[4], nC[4], lC[4];
    float carH[4] = {0, 0, 0, 0}, carN[4] = {0, 0, 0, 0};  // north link: mu*dh2, mu*dnl
    bool ok = true;
    if (r0 > 0) {
        ok = wait_row(r0 - 1);
        if (ok) waited = r0;
    }
    if (ok) {
        ok = wait_row(r0);
        if (ok) waited = r0 + 1;
    }
    if (!ok) {
        drain_and_fail();
        return;
    }
    {
        const float* P = row_ptr(r0);
        float ha[4], la[4];
        lds4(hC, P + kSt + x0);
        lds4(zC, P + kZ + x0);
        n4(nC, P);
        lds4(ha, P + kHa + x0);
        lds4(la, P + kLam + x0);
#pragma unroll
        for (int q = 0; q < 4; ++q) lC[q] = masked(ha[q], la[q]);
        if (r0 > 0) {  // the strip's north links, recomputed
            const float* U = row_ptr(r0 - 1);
            float hU[4], zU[4], nU[4], qU[4], lqU[4], haU[4], lhU[4], lU[4];
            lds4(hU, U + kSt + x0);
            lds4(zU, U + kZ + x0);
            n4(nU, U);
            lds4(qU, U + kSt + 2 * kBox + x0);
            lds4(lqU, U + kLam + 2 * kBox + x0);
            lds4(haU, U + kHa + x0);
            lds4(lhU, U + kLam + x0);
#pragma unroll
            for (int q = 0; q < 4; ++q) lU[q] = masked(haU[q], lhU[q]);
            if (act)
                north_carry<LIM>(hU, zU, nU, qU, lqU, lU, hC, zC, nC, lC, c, nx, s_half, T, k,
                                 carH, carN);
            release();
        }
    }

    // FP32 compensated sums of the rows' partials (lambda~ for the rain
    // gradient, mu n dq'/dn for the scale gradient), widened to FP64 once per warp
    float gr_s = 0.0f, gr_c = 0.0f, gs_s = 0.0f, gs_c = 0.0f;
    float gd_s = 0.0f, gd_c = 0.0f;  // land cover: drainage partials
    for (int r = r0; r < r1; ++r) {
        const size_t o = (size_t)r * ld + c;
        const bool has_s = (r + 1 < ny);
        if (has_s) {
            if (!wait_row(r + 1)) {
                drain_and_fail();
                return;
            }
            waited = r + 2;
        }
        const float* P = row_ptr(r);
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0}, lS[4] = {0, 0, 0, 0};
        float qxo[4], qyo[4], lqx[4], lqy[4];
        lds4(qxo, P + kSt + kBox + x0);
        lds4(qyo, P + kSt + 2 * kBox + x0);
        lds4(lqx, P + kLam + kBox + x0);
        lds4(lqy, P + kLam + 2 * kBox + x0);
        if (has_s) {
            const float* Q = row_ptr(r + 1);
            float ha[4], la[4];
            lds4(hS, Q + kSt + x0);
            lds4(zS, Q + kZ + x0);
            n4(nS, Q);
            lds4(ha, Q + kHa + x0);
            lds4(la, Q + kLam + x0);
#pragma unroll
            for (int q = 0; q < 4; ++q) lS[q] = masked(ha[q], la[q]);
        }
        // east neighbour of the lane's last cell and the span's west
        // neighbour, straight from the tile's halo
        const float hE = P[kSt + x0 + 4], zE = P[kZ + x0 + 4], nE = n1(P, x0 + 4);
        const float lE = masked(P[kHa + x0 + 4], P[kLam + x0 + 4]);
        const float nW = n1(P, 3);
        WestIn wi{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (lane == 0 && c0 > 0) {
            wi.h = P[kSt + 3]; wi.z = P[kZ + 3]; wi.n = nW;
            wi.qx = P[kSt + kBox + 3]; wi.lqx = P[kLam + kBox + 3];
            wi.l = masked(P[kHa + 3], P[kLam + 3]);
        }
        float lh[4], lx[4], ly[4], gnr[4];
        float gr_row = 0.0f, gs_row = 0.0f;
        float rwv[4] = {0, 0, 0, 0};
        if (LC) {
            float dfv[4], haC[4];
            const uint32_t wc = cls4(P);
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // the cells' runoff shares and drainage flags
                const float rv = __shfl_sync(0xffffffffu, lro, (int)(wc >> (8 * q)));
                const float dv = __shfl_sync(0xffffffffu, ldr, (int)(wc >> (8 * q)));
                rwv[q] = act ? rv : 0.0f;
                dfv[q] = act ? dv : 0.0f;
            }
            lds4(haC, P + kHa + x0);
            kahan_add(gd_s, gd_c, drain_row(lC, haC, dfv));
        }
        if (interior)
            adjoint_row<true, LIM, LC>(hC, zC, nC, lC, hS, zS, nS, lS, qxo, qyo, lqx, lqy, hE, zE,
                                       nE, lE, c0 > 0, wi, has_s, c, nx, lane, s, s_half, T, k,
                                       a.east_out, a.south_out, carH, carN, gr_row, gs_row, lh, lx,
                                       ly, gnr, rwv);
        else
            adjoint_row<false, LIM, LC>(hC, zC, nC, lC, hS, zS, nS, lS, qxo, qyo, lqx, lqy, hE, zE,
                                        nE, lE, c0 > 0, wi, has_s, c, nx, lane, s, s_half, T, k,
                                        a.east_out, a.south_out, carH, carN, gr_row, gs_row, lh, lx,
                                        ly, gnr, rwv);
        kahan_add(gr_s, gr_c, gr_row);
        kahan_add(gs_s, gs_c, gs_row);
        if (act) {
            store4(lout + o, lh);
            store4(lout + plane + o, lx);
            store4(lout + 2 * plane + o, ly);
            if (gn) {
                float g[4];
                lds4(g, P + kGn + x0);
#pragma unroll
                for (int q = 0; q < 4; ++q) g[q] += gnr[q];
                store4(gn + o, g);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hC[q] = hS[q]; zC[q] = zS[q]; nC[q] = nS[q]; lC[q] = lS[q];
        }
        release();
    }
    const int vslot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
    adjoint_partials(a.gpart, a.nslot, m, vslot, lane, gr_s, gr_c, gs_s, gs_c, pl.rdt,
                     1.0 / (double)s);
    if (LC) adjoint_drain_partial(a.gdpart, a.nslot, m, vslot, lane, gd_s, gd_c, pl.dt);
}

template <int WM, bool LC>
size_t adj_smem_bytes()
{
    (void)LC;  // the land-cover stage has the plain layout
    return 128 + 128 * ((8 * kNS * WM + 127) / 128) + (size_t)kNS * kStageBytes * WM;
}

template <int LIM, bool LC>
void launch_adjoint_tma_lim(const AdjTmaArgs& t, int members_per_cta, cudaStream_t s)
{
    const AdjArgs& a = t.a;
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4 && a.M >= 4) {
        static bool attr = false;
        const size_t shm = adj_smem_bytes<4, LC>();
        if (!attr) {
            cudaFuncSetAttribute(adjoint_tma_kernel<4, LIM, LC>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            attr = true;
        }
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        adjoint_tma_kernel<4, LIM, LC><<<grid, block, shm, s>>>(t);
    } else {
        const size_t shm = adj_smem_bytes<1, LC>();
        dim3 grid(a.M, spans, strips), block(32, 1);
        adjoint_tma_kernel<1, LIM, LC><<<grid, block, shm, s>>>(t);
    }
}

}  // namespace

void launch_adjoint_tma(const AdjTmaArgs& t, int members_per_cta, cudaStream_t s)
{
    if (t.a.rw)
        t.a.limiter ? launch_adjoint_tma_lim<1, true>(t, members_per_cta, s)
                    : launch_adjoint_tma_lim<0, true>(t, members_per_cta, s);
    else
        t.a.limiter ? launch_adjoint_tma_lim<1, false>(t, members_per_cta, s)
                    : launch_adjoint_tma_lim<0, false>(t, members_per_cta, s);
}

int adjoint_tma_box_cols() { return kBox; }

}  // namespace flood
