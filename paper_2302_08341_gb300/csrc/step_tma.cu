// TMA-staged variant of the fused local-inertial step (same arithmetic and
// results, bit for bit, as step_kernel.cu).
//
// Each warp owns one member's 128-column span of a strip of rows, as in the
// direct-load kernel, but its rows arrive through a ring of kNS shared-memory
// stages filled by the tensor memory accelerator: one 3-D tiled copy brings a
// row of h, qx and qy (136 columns: the span plus 4 halo columns each side,
// zero-filled past the grid's edges), another the same row of z and n.  Lane
// 0 keeps kNS - 1 rows in flight ahead of the row being computed, so the
// memory latency is covered by the warp's own pipeline instead of by register
// prefetch; the halo comes with the tile, so no scalar edge loads remain.
// Every mbarrier wait is bounded: on timeout the kernel records
// FLOOD_ERR_TIMEOUT in the error word, waits (bounded) for its own copies in
// flight, and returns.
#include <cudaTypedefs.h>

#include "march.cuh"
#include "tma.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;
constexpr int kNS = 4;                          // stages per warp
constexpr int kBox = kSpan + 8;                 // columns per tile row
constexpr int kStaticOff = 1664;                // bytes: z, n after h, qx, qy (128-aligned)
constexpr int kStageBytes = 2816;               // 128-aligned stage size
constexpr uint32_t kTx = kBox * 3 * 4 + kBox * 2 * 4;  // bytes landing per stage
constexpr int kZ = kStaticOff / 4;              // float offset of the z row in a stage
constexpr int kN = kZ + kBox;                   // float offset of the n row
constexpr long long kWaitBudget = 200000000LL;  // clock cycles (~0.1 s) before giving up

__device__ __forceinline__ void lds4(float (&v)[4], const float* p)
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int WM>
__global__ void __launch_bounds__(32 * WM, 20 / WM) step_tma_kernel(const __grid_constant__ TmaArgs t)
{
    extern __shared__ unsigned char smem_raw[];
    const StepArgs& a = t.a;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int m = blockIdx.x * WM + w;
    const int span = blockIdx.y;
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps; no block-wide barriers below
    if (*reinterpret_cast<volatile const int*>(a.err) & 2) return;  // an earlier wait gave up

    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    const uint32_t bar0 = smem_u32(base) + 8u * kNS * w;
    unsigned char* my_stages = base + 128 * ((8 * kNS * WM + 127) / 128) + kNS * kStageBytes * w;
    const uint32_t stage0 = smem_u32(my_stages);

    const int nx = a.nx, ny = a.ny, ld = a.ld;
    const size_t plane = a.plane;
    const size_t mstride = 3 * plane;
    // each warp is its own member here: the warp at the first span and strip owns its clock
    const MemberPlan pl = a.plan[m];
    if (!pl.active) return;
    float* __restrict__ dst = a.state + (size_t)((1 - pl.cur) * a.M + m) * mstride;
    float* ck = pl.ckpt >= 0 ? a.ckpt + ((size_t)pl.ckpt * a.M + m) * mstride : nullptr;

    FaceK k;
    k.gdt_dx = pl.gdt_dx;
    k.gdt = pl.gdt;
    k.dx_4dt = pl.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    const float dt_dx = pl.dt_dx;
    const float s = a.scale[m];
    const float s_half = 0.5f * s;
    const float dr = pl.dr;

    const int c = c0 + 4 * lane;
    const bool act = c < nx;
    const bool interior = (c + 4 < nx);
    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, ny);
    const int ra = r0 > 0 ? r0 - 1 : r0;   // first row loaded
    const int rb = min(r1 + 1, ny);        // one past the last row loaded
    const int plane0 = (pl.cur * a.M + m) * 3;

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
        mbar_arrive_expect_tx(bar, kTx);
        tma_load_3d(dsts, &t.state_map, c0 - 4, row, plane0, bar);
        tma_load_3d(dsts + kStaticOff, &t.static_map, c0 - 4, row, 0, bar);
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
    // recycle the stage of `row` for the next row in line
    auto release = [&](int row) {
        __syncwarp();
        if (issued < rb) {
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(issued);
            }
            ++issued;
        }
        (void)row;
    };
    int waited = ra;  // rows [ra, waited) have landed
    bool ok = true;
    auto drain_and_fail = [&]() {
        if (lane == 0) atomicOr(a.err, 2);
        for (int row = waited; row < issued; ++row) wait_row(row);  // bounded each
    };

    const int x0 = 4 + 4 * lane;  // this lane's first cell in a tile row
    float hC[4] = {0, 0, 0, 0}, zC[4] = {0, 0, 0, 0}, nC[4] = {0, 0, 0, 0};
    float qyN[4] = {0, 0, 0, 0};
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
        lds4(hC, P + x0);
        lds4(zC, P + kZ + x0);
        lds4(nC, P + kN + x0);
        if (r0 > 0) {
            const float* U = row_ptr(r0 - 1);
            float hU[4], zU[4], nU[4], qU[4];
            lds4(hU, U + x0);
            lds4(zU, U + kZ + x0);
            lds4(nU, U + kN + x0);
            lds4(qU, U + 2 * kBox + x0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                qyN[j] = (c + j < nx)
                             ? link_q(hU[j], zU[j], hC[j], zC[j], qU[j],
                                      __fmul_rn(s_half, __fadd_rn(nU[j], nC[j])), k)
                             : 0.0f;
            release(r0 - 1);
        }
    }

    float hmax = 0.0f;
    bool bad = false;
    float out_s = 0.0f, out_c = 0.0f, clamp = 0.0f;

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
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0};
        float qxo[4], qyo[4];
        lds4(qxo, P + kBox + x0);
        lds4(qyo, P + 2 * kBox + x0);
        if (has_s) {
            const float* Q = row_ptr(r + 1);
            lds4(hS, Q + x0);
            lds4(zS, Q + kZ + x0);
            lds4(nS, Q + kN + x0);
        }
        // east neighbour of the lane's last cell, straight from the tile
        const float hE = P[x0 + 4], zE = P[kZ + x0 + 4], nE = P[kN + x0 + 4];
        float qxE[4], qyS[4];
        if (interior)
            row_links<true>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                            a.east_out, a.south_out, qxE, qyS);
        else
            row_links<false>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                             a.east_out, a.south_out, qxE, qyS);
        float qW0 = __shfl_up_sync(0xffffffffu, qxE[3], 1);
        if (lane == 0) {
            qW0 = 0.0f;
            if (c0 > 0)  // the neighbouring span's last link, from the tile's halo
                qW0 = link_q(P[3], P[kZ + 3], hC[0], zC[0], P[kBox + 3],
                             __fmul_rn(s_half, __fadd_rn(P[kN + 3], nC[0])), k);
        }
        float hN[4];
        float hsum = 0.0f;
        if (interior)
            row_depths<true>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hsum, hN);
        else
            row_depths<false>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hsum, hN);
        bad |= !(hsum <= 3.0e38f);
        float ev = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c + j == nx - 1 && a.east_out) ev = qxE[j];
        if (!has_s && a.south_out)
            ev = __fadd_rn(ev, __fadd_rn(__fadd_rn(qyS[0], qyS[1]), __fadd_rn(qyS[2], qyS[3])));
        kahan_add(out_s, out_c, ev);
        if (act) {
            store4(dst + o, hN);
            store4(dst + plane + o, qxE);
            store4(dst + 2 * plane + o, qyS);
            if (ck) {
                store4(ck + o, hN);
                store4(ck + plane + o, qxE);
                store4(ck + 2 * plane + o, qyS);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            qyN[j] = qyS[j];
            hC[j] = hS[j];
            zC[j] = zS[j];
            nC[j] = nS[j];
        }
        release(r);
    }

    if (bad) atomicOr(a.err, 1);
    const unsigned hb = __reduce_max_sync(0xffffffffu, __float_as_uint(hmax) & 0x7fffffffu);
    double out_acc = (double)out_s - (double)out_c, clamp_acc = (double)clamp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        out_acc += __shfl_xor_sync(0xffffffffu, out_acc, off);
        clamp_acc += __shfl_xor_sync(0xffffffffu, clamp_acc, off);
    }
    if (lane == 0) {
        atomicMax(&a.ms_out[m].hmax_bits, hb);
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            const int slot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
            double* v = a.vacc + ((size_t)m * a.nslot + slot) * 2;
            v[0] += out_acc * pl.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
    }
}

template <int WM>
size_t tma_smem_bytes()
{
    return 128 + 128 * ((8 * kNS * WM + 127) / 128) + (size_t)kNS * kStageBytes * WM;
}

}  // namespace

int encode_map_3d(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                  uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t b0, uint32_t b1, uint32_t b2)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

int tma_box_cols() { return kBox; }

int launch_step_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s)
{
    const StepArgs& a = t.a;
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        static bool attr = false;
        const size_t shm = tma_smem_bytes<4>();
        if (!attr) {
            cudaFuncSetAttribute(step_tma_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            attr = true;
        }
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        step_tma_kernel<4><<<grid, block, shm, s>>>(t);
    } else {
        const size_t shm = tma_smem_bytes<1>();
        dim3 grid(a.M, spans, strips), block(32, 1);
        step_tma_kernel<1><<<grid, block, shm, s>>>(t);
    }
    return 0;
}

}  // namespace flood
