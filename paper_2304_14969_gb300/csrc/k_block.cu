// Dense k-qubit block (SIMT): psi <- U psi on qubits Q, |Q| = k <= 7.
//
// Table I of arXiv 2304.14969 ("coalesced gates executed with a single
// traversal"): a block of gates multiplied into one 2^k x 2^k unitary on the
// host costs one HBM read+write of the ket. A CTA stages 32 groups (the 2^k
// amplitudes that differ only in Q) in shared memory with U, then each
// thread forms 4 output rows of one group. Group g's base index has zeros
// at Q; consecutive groups are consecutive in the lowest non-Q bits, so a
// warp's 32 loads of one row element are contiguous when qubit 0..4 are not
// in Q.
#include <algorithm>
#include <cuda_runtime.h>

#include "qsim_internal.h"

namespace qs {

template <typename R> struct BV2;
template <> struct BV2<float> { using T = float2; };
template <> struct BV2<double> { using T = double2; };

struct BlockSpec {
    int k;
    int q[8];          // physical bit of block index bit b
    InsSpec ins;       // sorted Q for group expansion
};

static const int kGroups = 32;

template <typename R>
__global__ void __launch_bounds__(256) k_block_simt(typename BV2<R>::T *__restrict__ a, uint64_t ngroups,
                                                    BlockSpec bs, const typename BV2<R>::T *__restrict__ Ug,
                                                    int u_in_smem)
{
    using V = typename BV2<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = bs.k, D = 1 << k;
    V *U = (V *)smraw;                                // D*D if u_in_smem
    V *vin = U + (u_in_smem ? D * D : 0);             // [D][kGroups]
    if (u_in_smem)
        for (int i = threadIdx.x; i < D * D; i += blockDim.x) U[i] = Ug[i];
    const V *Ur = u_in_smem ? U : Ug;

    // spread of block index l into physical index bits
    auto spread = [&](int l) {
        uint64_t o = 0;
        for (int b = 0; b < k; b++)
            if ((l >> b) & 1) o |= 1ull << bs.q[b];
        return o;
    };
    const int RB = 4;                                  // rows per thread
    const int rows_per_pass = (blockDim.x / kGroups) * RB;

    for (uint64_t g0 = (uint64_t)blockIdx.x * kGroups; g0 < ngroups; g0 += (uint64_t)gridDim.x * kGroups) {
        __syncthreads();
        // gather: element (l, gl) -> vin[l * kGroups + gl]
        for (int e = threadIdx.x; e < D * kGroups; e += blockDim.x) {
            int l = e / kGroups, gl = e % kGroups;
            uint64_t g = g0 + gl;
            V v;
            v.x = 0;
            v.y = 0;
            if (g < ngroups) {
                uint64_t base = g;
                for (int j = 0; j < bs.ins.npos; j++) {
                    int p = bs.ins.pos[j];
                    base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
                }
                v = a[base | spread(l)];
            }
            vin[e] = v;
        }
        __syncthreads();
        int gl = threadIdx.x % kGroups;
        uint64_t g = g0 + gl;
        uint64_t base = g;
        for (int j = 0; j < bs.ins.npos; j++) {
            int p = bs.ins.pos[j];
            base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
        }
        for (int r0 = (threadIdx.x / kGroups) * RB; r0 < D; r0 += rows_per_pass) {
            R orr[RB], oi[RB];
#pragma unroll
            for (int j = 0; j < RB; j++) { orr[j] = 0; oi[j] = 0; }
            for (int c = 0; c < D; c++) {
                V x = vin[c * kGroups + gl];
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    if (r0 + j < D) {
                        V u = Ur[(r0 + j) * D + c];
                        orr[j] = fma(u.x, x.x, orr[j]);
                        orr[j] = fma(-u.y, x.y, orr[j]);
                        oi[j] = fma(u.x, x.y, oi[j]);
                        oi[j] = fma(u.y, x.x, oi[j]);
                    }
                }
            }
            if (g < ngroups) {
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    if (r0 + j < D) {
                        V o;
                        o.x = orr[j];
                        o.y = oi[j];
                        a[base | spread(r0 + j)] = o;
                    }
                }
            }
        }
    }
}

cudaError_t launch_fused_simt(qsim_state *s, int k, const int *phys, const cd *u)
{
    BlockSpec bs;
    bs.k = k;
    std::vector<int> pos;
    for (int b = 0; b < k; b++) {
        bs.q[b] = phys[b];
        pos.push_back(phys[b]);
    }
    std::sort(pos.begin(), pos.end());
    bs.ins.npos = k;
    for (int b = 0; b < k; b++) bs.ins.pos[b] = pos[b];
    const int D = 1 << k;
    const size_t es = s->dt == QSIM_C64 ? 8 : 16;
    // upload U in the state's precision
    void *dU = nullptr;
    cudaError_t e = cudaMallocAsync(&dU, (size_t)D * D * es, s->stream);
    if (e != cudaSuccess) return e;
    std::vector<float2> uf;
    std::vector<double2> ud;
    if (s->dt == QSIM_C64) {
        uf.resize((size_t)D * D);
        for (size_t i = 0; i < uf.size(); i++) uf[i] = make_float2((float)u[i].real(), (float)u[i].imag());
        e = cudaMemcpyAsync(dU, uf.data(), uf.size() * es, cudaMemcpyHostToDevice, s->stream);
    } else {
        ud.resize((size_t)D * D);
        for (size_t i = 0; i < ud.size(); i++) ud[i] = make_double2(u[i].real(), u[i].imag());
        e = cudaMemcpyAsync(dU, ud.data(), ud.size() * es, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) {
        size_t usz = (size_t)D * D * es;
        int in_smem = usz <= 128 * 1024;
        size_t smem = (in_smem ? usz : 0) + (size_t)D * kGroups * es;
        uint64_t ngroups = s->N() >> k;
        int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((ngroups + kGroups - 1) / kGroups, 152 * 4));
        if (s->dt == QSIM_C64) {
            cudaFuncSetAttribute(k_block_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_block_simt<float><<<blocks, 256, smem, s->stream>>>((float2 *)s->amps, ngroups, bs, (const float2 *)dU,
                                                                 in_smem);
        } else {
            cudaFuncSetAttribute(k_block_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_block_simt<double><<<blocks, 256, smem, s->stream>>>((double2 *)s->amps, ngroups, bs,
                                                                  (const double2 *)dU, in_smem);
        }
        e = cudaGetLastError();
    }
    cudaStreamSynchronize(s->stream);  // host staging vectors die at return
    cudaFreeAsync(dU, s->stream);
    return e;
}

}  // namespace qs
