// hc_batch.cu -- the batched kernels of a parameter sweep (2D, HC_FP32_REFINED).
//
// The members of a size class (one grid size, any c, D, gamma, dt, r, S, m0,
// domain lengths) advance together: every pass of the step (Algorithm 1's
// loop body: the FP32 first residual, the inner CG iterations, the
// double-float mid-step residual, the FP64 refinement residual, the split
// step) is ONE launch over all members, blockIdx.y = member.  Each member
// keeps its own solve state, so its CG and refinement loops stop on their own
// tolerances: a member that has finished a loop returns at once from that
// loop's later launches.  The graph's loop conditions are the OR over the
// members (batch_flags), so a loop runs until its slowest member is done.
// The per-member work is the single-problem kernels' bodies unchanged.
#include "hc_kernels.cuh"

namespace hc {

namespace {

// The FP32 gradient and divergence passes take the class tile (CTAs of up to
// 1024 threads), the heat pass at most 512 threads (gfn, col_narrow).

// ------------------------------------------------------------------ FP32 first residual
__global__ void __launch_bounds__(1024, 1) kb_first_grad(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_grad_body<float, double, CG_PLAIN>(c.gf, c.p64, nullptr, nullptr, nullptr, c.G32,
                                         c.G32 + c.ns, c.st, 0);
}
template <int NV>
__global__ void __launch_bounds__(512) kb_first_apply(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  row_apply_body<float, float, false, NV>(c.gf, c.G32, c.G32 + c.ns, c.mx, c.my, c.rf, c.G32,
                                          c.G32 + c.ns, nullptr);
}
__global__ void __launch_bounds__(1024, 1) kb_first_div(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_div_body<float, CD_RESID_FIRST>(c.gf, c.G32, c.G32 + c.ns, nullptr, c.b32, nullptr, c.r32,
                                      c.x32, c.st);
}

// ------------------------------------------------------------------ inner FP32 CG iteration
__global__ void __launch_bounds__(1024, 1) kb_cg_grad(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_grad_body<float, float, CG_DUPDATE>(c.gf, (cx<float>*)nullptr, c.r32, c.d32, nullptr, c.G32,
                                          c.G32 + c.ns, c.st, 1);
}
template <int NV>
__global__ void __launch_bounds__(512) kb_cg_apply(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  row_apply_body<float, float, true, NV>(c.gf, c.G32, c.G32 + c.ns, c.mx, c.my, c.rf, c.G32,
                                         c.G32 + c.ns, c.st);
}
__global__ void __launch_bounds__(1024, 1) kb_cg_div(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_div_body<float, CD_CG>(c.gf, c.G32, c.G32 + c.ns, c.d32, nullptr, c.q32, nullptr, nullptr,
                             c.st);
}
__global__ void __launch_bounds__(256, 4) kb_cg_update(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  cg_update_body<float>(c.gf, c.x32, c.r32, c.d32, c.q32, c.st);
}

// ------------------------------------------------------------------ mid-step residual (double-float)
// Only members whose first sweep ran have it pending (mid_phase); the last CTA
// of the divergence pass clears the flag, after every CTA has passed this test.
__global__ void __launch_bounds__(512) kb_mid_grad(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (!c.st->mid_phase) return;
  cx<df64>* G = reinterpret_cast<cx<df64>*>(c.G64);
  col_grad_body<df64, double, CG_ADDDELTA>(c.gq, c.p64, nullptr, nullptr, c.x32, G, G + c.ns, c.st,
                                           0);
}
__global__ void __launch_bounds__(512) kb_mid_apply(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (!c.st->mid_phase) return;
  cx<df64>* G = reinterpret_cast<cx<df64>*>(c.G64);
  row_apply_body<df64, float, false, 1>(c.gq, G, G + c.ns, c.mx, c.my, c.rf, G, G + c.ns, nullptr);
}
__global__ void __launch_bounds__(512) kb_mid_div(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (!c.st->mid_phase) return;
  cx<df64>* G = reinterpret_cast<cx<df64>*>(c.G64);
  col_div_body<df64, CD_RESID_REFINE>(c.gq, G, G + c.ns, nullptr, c.bq, nullptr, c.r32, c.x32,
                                      c.st);
}

// ------------------------------------------------------------------ FP64 refinement residual
// Only members whose refinement loop is still open (the last CTA of the
// divergence pass decides, after every CTA has passed this test).
__global__ void __launch_bounds__(512) kb_res_grad(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (c.st->outer_done) return;
  col_grad_body<double, double, CG_ADDDELTA>(c.gd, c.p64, nullptr, nullptr, c.x32, c.G64,
                                             c.G64 + c.ns, c.st, 0);
}
__global__ void __launch_bounds__(512) kb_res_apply(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (c.st->outer_done) return;
  row_apply_body<double, float, false, 1>(c.gd, c.G64, c.G64 + c.ns, c.mx, c.my, c.rf, c.G64,
                                          c.G64 + c.ns, nullptr);
}
__global__ void __launch_bounds__(512) kb_res_div(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  if (c.st->outer_done) return;
  col_div_body<double, CD_RESID_REFINE>(c.gd, c.G64, c.G64 + c.ns, nullptr, c.b64, c.r64, c.r32,
                                        c.x32, c.st);
}

// ------------------------------------------------------------------ split step
__global__ void __launch_bounds__(1024, 1) kb_split_grad(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_grad_body<float, double, CG_PLAIN>(c.gf, c.p64, nullptr, nullptr, nullptr, c.G32,
                                         c.G32 + c.ns, c.st, 0);
}
__global__ void __launch_bounds__(512) kb_split_row(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  row_split_body<float>(c.gf, c.G32, c.G32 + c.ns, c.mx, c.my, c.rf, c.G32, c.G32 + c.ns, c.cf,
                        c.st);
}
__global__ void __launch_bounds__(512) kb_split_heat(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  col_heat_body<float>(c.gfn, c.G32, c.G32 + c.ns, c.st);
}
__global__ void __launch_bounds__(512) kb_split_c2r(const BInst* bi) {
  const BInst& c = bi[blockIdx.y];
  row_c2r_body<float>(c.gf, c.G32, c.G32 + c.ns, c.mx, c.my, c.st, 1);
}

// ------------------------------------------------------------------ bookkeeping
// One thread per member.  The refinement loop opens for every member (all are
// refined), so the class's outer condition is set to 1 here.
__global__ void kb_step_begin(const BInst* bi, int nb, int npts, cudaGraphConditionalHandle h_outer) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) step_begin_body(bi[b].st, npts);
  if (b == 0) cudaGraphSetConditional(h_outer, 1u);
}
// The split step and step end close the step: 5 kernels of the class.
__global__ void kb_step_end(const BInst* bi, int nb, long long* launches) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) step_end_body(bi[b].st, 1);
  if (b == 0) *launches += 5;
}
// Loop conditions of the class: OR over members, by one warp.  BF_FIRST (after
// the first residual): h1 = some member runs a first inner solve, h2 = some
// member has the mid-step residual pending.  BF_LOOP (after a CG iteration or
// the mid-step residual): h1 = some member's inner solve is still running.
// BF_REFINE (after an FP64 residual): h1 as BF_LOOP, h2 = some member's
// refinement loop is still open.  `kernels` = launches of the segment this
// kernel closes, itself included.
__global__ void kb_flags(const BInst* bi, int nb, int kind, cudaGraphConditionalHandle h1,
                         cudaGraphConditionalHandle h2, long long* launches, int kernels) {
  bool a = false, b = false;
  for (int i = threadIdx.x; i < nb; i += 32) {
    const SolveState* st = bi[i].st;
    a = a || !st->done;
    if (kind == BF_FIRST) b = b || st->mid_phase;
    if (kind == BF_REFINE) b = b || !st->outer_done;
  }
  a = __any_sync(0xffffffffu, a);
  b = __any_sync(0xffffffffu, b);
  if (threadIdx.x == 0) {
    cudaGraphSetConditional(h1, a ? 1u : 0u);
    if (kind != BF_LOOP && h2) cudaGraphSetConditional(h2, b ? 1u : 0u);
    *launches += kernels;
  }
}

dim3 row_grid(const Geo<float>& g, int nb) { return dim3(g.ny >> g.lrpc, nb); }
template <typename T>
dim3 col_grid(const Geo<T>& g, int nb) { return dim3(g.H >> g.ltc, nb); }

}  // namespace

void batch_step_begin(const BInst* bi, const BShape& sh, cudaGraphConditionalHandle h_outer,
                      cudaStream_t s) {
  kb_step_begin<<<(sh.nb + 127) / 128, 128, 0, s>>>(bi, sh.nb, sh.gf.nx * sh.gf.ny, h_outer);
}

// The FP32 row pass of the operator apply takes two rows per thread when the
// geometry puts two or more rows in a CTA, as row_apply does.
void batch_first_resid(const BInst* bi, const BShape& sh, cudaStream_t s) {
  const Geo<float>& g = sh.gf;
  kb_first_grad<<<col_grid(g, sh.nb), col_threads(g), col_smem(g, 2), s>>>(bi);
  const size_t sm = row_smem(g) + (size_t)3 * g.rpc * g.nx * sizeof(float);
  if (g.rpc >= 2)
    kb_first_apply<2><<<row_grid(g, sh.nb), row_threads(g) >> 1, sm, s>>>(bi);
  else
    kb_first_apply<1><<<row_grid(g, sh.nb), row_threads(g), sm, s>>>(bi);
  kb_first_div<<<col_grid(g, sh.nb), col_threads(g), col_smem(g, 2), s>>>(bi);
}

void batch_cg_iter(const BInst* bi, const BShape& sh, cudaStream_t s) {
  const Geo<float>& g = sh.gf;
  kb_cg_grad<<<col_grid(g, sh.nb), col_threads(g), col_smem(g, 2), s>>>(bi);
  const size_t sm = row_smem(g) + (size_t)3 * g.rpc * g.nx * sizeof(float);
  if (g.rpc >= 2)
    kb_cg_apply<2><<<row_grid(g, sh.nb), row_threads(g) >> 1, sm, s>>>(bi);
  else
    kb_cg_apply<1><<<row_grid(g, sh.nb), row_threads(g), sm, s>>>(bi);
  kb_cg_div<<<col_grid(g, sh.nb), col_threads(g), col_smem(g, 2), s>>>(bi);
  kb_cg_update<<<dim3(upd_blocks((size_t)g.ny * g.H), sh.nb), 256, 0, s>>>(bi);
}

void batch_mid_resid(const BInst* bi, const BShape& sh, cudaStream_t s) {
  const Geo<df64>& q = sh.gq;
  kb_mid_grad<<<col_grid(q, sh.nb), col_threads(q), col_smem(q, 2), s>>>(bi);
  const size_t sm = row_smem(q) + (size_t)3 * q.rpc * q.nx * sizeof(float);
  kb_mid_apply<<<dim3(q.ny >> q.lrpc, sh.nb), row_threads(q), sm, s>>>(bi);
  kb_mid_div<<<col_grid(q, sh.nb), col_threads(q), col_smem(q, 2), s>>>(bi);
}

void batch_refine_resid(const BInst* bi, const BShape& sh, cudaStream_t s) {
  const Geo<double>& d = sh.gd;
  kb_res_grad<<<col_grid(d, sh.nb), col_threads(d), col_smem(d, 2), s>>>(bi);
  const size_t sm = row_smem(d) + (size_t)3 * d.rpc * d.nx * sizeof(float);
  kb_res_apply<<<dim3(d.ny >> d.lrpc, sh.nb), row_threads(d), sm, s>>>(bi);
  kb_res_div<<<col_grid(d, sh.nb), col_threads(d), col_smem(d, 2), s>>>(bi);
}

void batch_split(const BInst* bi, const BShape& sh, cudaStream_t s) {
  const Geo<float>& g = sh.gf;
  const Geo<float>& gn = sh.gfn;
  kb_split_grad<<<col_grid(g, sh.nb), col_threads(g), col_smem(g, 2), s>>>(bi);
  kb_split_row<<<row_grid(g, sh.nb), row_threads(g), row_split_smem(g), s>>>(bi);
  kb_split_heat<<<col_grid(gn, sh.nb), col_threads(gn), col_smem(gn, 2), s>>>(bi);
  kb_split_c2r<<<row_grid(g, sh.nb), row_threads(g), row_smem(g), s>>>(bi);
}

void batch_step_end(const BInst* bi, const BShape& sh, long long* launches, cudaStream_t s) {
  kb_step_end<<<(sh.nb + 127) / 128, 128, 0, s>>>(bi, sh.nb, launches);
}

void batch_flags(const BInst* bi, const BShape& sh, int kind, cudaGraphConditionalHandle h1,
                 cudaGraphConditionalHandle h2, long long* launches, int kernels, cudaStream_t s) {
  kb_flags<<<1, 32, 0, s>>>(bi, sh.nb, kind, h1, h2, launches, kernels);
}

void set_smem_limits_batch() {
  allow_smem(kb_first_grad);
  allow_smem(kb_first_apply<1>);
  allow_smem(kb_first_apply<2>);
  allow_smem(kb_first_div);
  allow_smem(kb_cg_grad);
  allow_smem(kb_cg_apply<1>);
  allow_smem(kb_cg_apply<2>);
  allow_smem(kb_cg_div);
  allow_smem(kb_mid_grad);
  allow_smem(kb_mid_apply);
  allow_smem(kb_mid_div);
  allow_smem(kb_res_grad);
  allow_smem(kb_res_apply);
  allow_smem(kb_res_div);
  allow_smem(kb_split_grad);
  allow_smem(kb_split_row);
  allow_smem(kb_split_heat);
  allow_smem(kb_split_c2r);
}

}  // namespace hc
