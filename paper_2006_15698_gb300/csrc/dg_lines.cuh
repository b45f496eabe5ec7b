// dg_lines.cuh -- the float form's single-mesh RK stage as a z-marching
// column kernel with one thread per z node line.  Included by dg_kernels.cuh
// (inside namespace dg), after dg_column.cuh, whose slot layout, prefetch,
// traces and flux routines it shares.
//
// As in column_stage_kernel, a CTA walks a column of TX x TY elements up a
// chunk of z layers and the layers ahead are staged in a ring of shared-
// memory slots by cp.async.  Here a thread owns the N nodes
// (i, j, 0..N-1) of one element of the layer, so all work along z stays in
// its registers: the z fluxes of its nodes and their weak z-derivative, the
// traces at the two z ends of its line and the z interface flux above it
// (kept as the next layer's -z face flux).  Per layer:
//
//   P  every thread: Euler fluxes (Eq. 2-3) of its nodes, x and y fluxes ->
//      shared memory as x and y node lines; the z interface flux above its
//      line (local Lax-Friedrichs, Sec. II.B) from its own +z trace and the
//      -z trace of the line above in the next slot;
//      interface tasks: the local Lax-Friedrichs flux at every x and y face
//      point of the layer, each interface once, from the traces of the
//      staged node lines on both sides (a neighbour column's line read
//      through L2) -> shared memory
//   G  every thread: weak derivative, lift of the six face fluxes and the
//      stage update of its nodes -> DRAM
//
// Traces, interface fluxes, node fluxes, the derivative sums and the update
// use the same functions in the same operation order as column_stage_kernel,
// so the two kernels give the same floats.
#pragma once

// Column cross-sections per N (= p + 1): one thread per z line, 64 to 256
// threads per CTA (measured on GB300; wider ones lose occupancy to shared
// memory and registers).  NS: slots in the ring of staged layers (3: the
// layer two ahead is fetched during a whole layer; 2: during the second
// phase only, less shared memory).  SWZ: swizzled slot layout (slot_pos).
// UT: the interface-task loop unrolled (more independent work per thread,
// more registers).  RC: the layer copied row by row (pays where a row is
// many copies per thread).  PFN: the neighbour columns' elements of the next
// layer prefetched into L2.  PL1: the current layer's neighbour-column
// elements prefetched into L1 before the node fluxes (measured on GB300: 2 %
// faster at p = 2, 0.5-5 % slower at p = 1 and 3..6; PFN on top of it at
// p = 2: 1.6 % slower).  RPAD: floats of padding
// after every element row of a slot, so that the rows of one x-interface
// task batch fall into different banks (where a row is a multiple of 32
// floats).
template <int N, int V>
struct LineShape;
struct LineDefaults {
    static constexpr bool SWZ = false, UT = false, RC = false, PFN = false, PL1 = false;
    static constexpr int NS = 3, RPAD = 0;
    // resident CTAs per SM the batched kernel must allow (its registers then
    // match the single-mesh kernel's; 0: no bound)
    static constexpr int BMINB = 0;
};
template <> struct LineShape<1, 0> : LineDefaults { static constexpr int TX = 16, TY = 16, NS = 2, RPAD = 1; };
template <> struct LineShape<2, 0> : LineDefaults { static constexpr int TX = 8, TY = 8, NS = 2, RPAD = 8, BMINB = 2; };
template <> struct LineShape<3, 0> : LineDefaults {
    static constexpr int TX = 4, TY = 4, NS = 2, BMINB = 3;
    static constexpr bool PL1 = true;
};
template <> struct LineShape<4, 0> : LineDefaults {
    static constexpr int TX = 2, TY = 2, NS = 2;
    static constexpr bool SWZ = true, UT = true, PFN = true;
};
template <> struct LineShape<5, 0> : LineDefaults { static constexpr int TX = 3, TY = 2, NS = 2; };
template <> struct LineShape<6, 0> : LineDefaults {
    static constexpr int TX = 3, TY = 1;
    static constexpr bool UT = true;
};
template <> struct LineShape<7, 0> : LineDefaults {
    static constexpr int TX = 2, TY = 1;
    static constexpr bool RC = true;
};

template <int N, int TX, int TY, int NS = 3, int RPAD = 0>
struct LineTile {
    using CT = ColTile<N, TX, TY>;  // element layout in a slot, prefetch units
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int EPB = TX * TY;
    static constexpr int THREADS = ((EPB * N2 + 31) / 32) * 32;
    // fluxes [x, y][NF][N3] as node lines; element stride = N^2 (mod 32), so
    // that the N^2 threads of consecutive elements store to consecutive banks
    static constexpr int FSTR = 2 * NF * N3 + ((N2 - (2 * NF * N3) % 32) % 32 + 32) % 32;
    // x, y face fluxes [2][NF][N2][(-,+)]; element stride = 2N (mod 32)
    // (even), so that the N (-,+) pairs each element reads at a time fall into
    // consecutive banks for consecutive elements (N = 4: the column layout's)
    static constexpr int HSTR =
        N == 4 ? CT::HSTR : 4 * NF * N2 + ((2 * N - (4 * NF * N2) % 32) % 32 + 32) % 32;
    static constexpr int FREG = (EPB * FSTR + 3) / 4 * 4;  // regions in 16-byte multiples
    static constexpr int HREG = (EPB * HSTR + 3) / 4 * 4;
    // a slot: [NF][TY] element rows of TX elements (ESTR apart), RSTR apart
    static constexpr int RSTR = TX * CT::ESTR + RPAD;
    static constexpr int QSLOT = (NF * TY * RSTR + 3) / 4 * 4;
    static constexpr size_t FLOATS = (size_t)NS * QSLOT + (size_t)FREG + (size_t)HREG + CT::OPSF;
    // offset of field n of slot element el (= b * TX + a)
    __device__ static constexpr int eoff(int n, int el)
    {
        if constexpr (RPAD == 0) return (n * EPB + el) * CT::ESTR;
        else return (n * TY + el / TX) * RSTR + (el % TX) * CT::ESTR;
    }
    static constexpr size_t BYTES = FLOATS * sizeof(float);
    static constexpr int XT = (TX + 1) * TY * N2, YT = (TY + 1) * TX * N2;
};

// trace of a staged node line (element el of the slot) at one end; base is
// the line's first node (line_base)
template <class LT, int N, int DIR, bool SWZ>
__device__ __forceinline__ void slot_trace(const float *slot, int el, int base, const float *l,
                                           float q[NF])
{
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? N : N * N);
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        const float *e = slot + LT::eoff(n, el);
        float v[N];
        if constexpr (DIR == 0) {
            load_line<N>(e + slot_pos<N, SWZ>(base), v);   // an x line is one 16-byte unit
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = e[slot_pos<N, SWZ>(base + c * stride)];
        }
        q[n] = line_dot<N>(l, v);
    }
}

// x (DIR 0) or y (DIR 1) interface a in [0, len] of row r at face point pt,
// both traces from node lines (staged, or the neighbour column's in DRAM/L2)
template <class LT, int N, int TX, int TY, int DIR, typename Ix, bool SWZ>
__device__ __forceinline__ void slot_interface(const float *__restrict__ Qin, const float *slot,
                                               float *sH, const Geo &g, const float *lm,
                                               const float *lp, float gamma, float gm1, int a,
                                               int r, int len, Ix e_lo, Ix e_hi, int pt)
{
    constexpr int N2 = LT::N2;
    const int base = line_base<N, DIR>(pt % N, pt / N);
    auto local = [&](int c) { return DIR == 0 ? r * TX + c : c * TX + r; };
    float qL[NF], qR[NF];
    if (a == 0) global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_lo, base, lp, qL);
    else slot_trace<LT, N, DIR, SWZ>(slot, local(a - 1), base, lp, qL);
    if (a == len) global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_hi, base, lm, qR);
    else slot_trace<LT, N, DIR, SWZ>(slot, local(a), base, lm, qR);
    float f[NF];
    lf_flux2_f<DIR>(qL, qR, gamma, gm1, f);
    if (a > 0) {
        float *h = sH + (size_t)local(a - 1) * LT::HSTR + (DIR * NF * N2 + pt) * 2 + 1;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
    if (a < len) {
        float *h = sH + (size_t)local(a) * LT::HSTR + (DIR * NF * N2 + pt) * 2 + 0;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
}

// The stage over one mesh: one CTA per (column, z chunk); MODE and Ix as for
// column_stage_kernel.  HALO: the mesh is a z slab (g.zlo, g.zhi set), its
// first and last layers' outer faces read the neighbours' traces (a
// compile-time switch, so that a periodic mesh's kernel carries none of that
// code).  The body (dg_line_body.inc) is shared with batched_line_kernel.
template <int N, int V, int MODE, typename Ix, bool HALO>
__global__ void __launch_bounds__(
    LineTile<N, LineShape<N, V>::TX, LineShape<N, V>::TY, LineShape<N, V>::NS,
             LineShape<N, V>::RPAD>::THREADS)
    line_stage_kernel(const float *__restrict__ Qin, float *__restrict__ Out,
                      float *__restrict__ dQ, const Ops<float> T, const Geo g, float A, float B,
                      const double *__restrict__ dt, int zchunk)
{
    const unsigned block = blockIdx.x;
#include "dg_line_body.inc"
}

// The stage over the instances of one degree of a batch: one CTA per work
// item (instance, column, z chunk), the body of line_stage_kernel
// (dg_line_body.inc) on the instance's arrays, so an instance's floats are
// those of the same mesh stepped alone.  parity 0: the stage reads Q and
// writes the second state Qt; 1: the reverse.
template <int N, int MODE, typename Ix>
__global__ void __launch_bounds__(
    LineTile<N, LineShape<N, 0>::TX, LineShape<N, 0>::TY, LineShape<N, 0>::NS,
             LineShape<N, 0>::RPAD>::THREADS, LineShape<N, 0>::BMINB)
    batched_line_kernel(const LineItem *__restrict__ items, const InstDev *__restrict__ inst,
                        int parity, float A, float B)
{
    // the instance's geometry staged in shared memory: the body reads it
    // where the single-mesh kernel reads its parameter bank, without holding
    // it in registers
    __shared__ Geo sg;
    const LineItem it = items[blockIdx.x];
    const InstDev *I = inst + it.inst;
    if (threadIdx.x == 0) sg = I->g;
    __syncthreads();
    constexpr int V = 0;
    constexpr bool HALO = false;
    const float *__restrict__ Qin = parity ? I->Qt : I->Q;
    float *__restrict__ Out = parity ? I->Q : I->Qt;
    float *__restrict__ dQ = I->dQ;
    const Ops<float> &T = I->T;
    const Geo &g = sg;
    const double *__restrict__ dt = I->dt;
    const int zchunk = it.zchunk;
    const unsigned block = (unsigned)it.block;
#include "dg_line_body.inc"
}
