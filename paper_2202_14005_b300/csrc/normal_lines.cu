// Fused SENSE normal operator for Cartesian line masks: plan tables and launcher (the kernel
// template is in normal_lines.cuh).
#include <algorithm>
#include <cmath>
#include <vector>

#include "normal_lines.cuh"

using namespace nl;

namespace {

// (Q, P) factorisations with a compiled kernel: W = 64, 128, 232, 256, 320, 368.
struct QP { int Q, P; };
const QP kSupported[] = {{8, 8}, {8, 16}, {8, 29}, {16, 16}, {16, 20}, {16, 23}};

NLKernel pick_kernel(int Q, int P, int jmax, int mode, int ns) {
  if (Q == 8) return pick_q8(P, jmax, mode, ns);
  if (Q == 16) return pick_q16(P, jmax, mode, ns);
  return nullptr;
}

}  // namespace

int build_lines_tables(sense_plan pl) {
  LinesTables& T = pl->lines;
  T = LinesTables();
  if (!pl->mask_is_lines) return SENSE_OK;
  const int W = pl->W;
  int Q = 0, P = 0;
  for (const QP& c : kSupported)  // prefer the largest Q (more coils per warp in phase B)
    if (c.Q * c.P == W && c.Q > Q) { Q = c.Q; P = c.P; }
  if (!Q) return SENSE_OK;  // generic path
  const int HP = (P - 1) / 2;
  const int RQ = (HP + 1) / 2;
  std::vector<std::vector<int>> slots(Q);
  std::vector<float> mplain(W);
  for (int k = 0; k < W; ++k) mplain[k] = pl->mask_h[(k + W / 2) % W];
  for (int k1 = 0; k1 < Q; ++k1)
    for (int k2 = 0; k2 < P; ++k2)
      if (mplain[k1 + Q * k2] != 0.f) slots[k1].push_back(k2);
  int J = 1;
  for (auto& s : slots) J = std::max<int>(J, (int)s.size());
  int JMAX = 0;
  for (int c : kJmax)
    if (!JMAX && J <= c) JMAX = c;
  if (!JMAX) return SENSE_OK;  // too dense for the pruned kernel: generic path
  int kstride = J * RQ;
  if (kstride % 2 == 0) kstride += 1;  // odd quad stride spreads k1 rows over banks
  std::vector<float4> coef((size_t)Q * kstride, make_float4(0, 0, 0, 0));
  std::vector<float2> tw((size_t)Q * P);
  std::vector<float> wt((size_t)Q * J, 0.f), sgn((size_t)Q * J, 0.f), af((size_t)Q * J, 0.f);
  std::vector<int> akx((size_t)Q * J, 0), cols;
  for (int kx = 0; kx < W; ++kx)
    if (pl->mask_h[kx] != 0.f) cols.push_back(kx);
  const double twopi = 2.0 * M_PI;
  for (int k1 = 0; k1 < Q; ++k1) {
    for (int t = 0; t < P; ++t) {
      const double ang = -twopi * (double)t * k1 / W;
      tw[(size_t)k1 * P + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
    for (int j = 0; j < (int)slots[k1].size(); ++j) {
      const int k2 = slots[k1][j];
      const double m = mplain[k1 + Q * k2];
      wt[(size_t)k1 * J + j] = (float)(m * m / W);
      sgn[(size_t)k1 * J + j] = (k2 & 1) ? -1.f : 1.f;
      const int k = k1 + Q * k2;  // plain frequency; its centred column is (k + W/2) mod W
      akx[(size_t)k1 * J + j] = (k + W / 2) % W;
      af[(size_t)k1 * J + j] = (float)(((k & 1) ? -1.0 : 1.0) / std::sqrt((double)W));
      for (int q = 0; q < RQ; ++q) {
        const int t = 2 * q + 1;
        float4 v = make_float4(0, 0, 0, 0);
        const double a0 = twopi * (double)((t * k2) % P) / P;
        v.x = (float)cos(a0);
        v.y = (float)sin(a0);
        if (t + 1 <= HP) {
          const double a1 = twopi * (double)(((t + 1) * k2) % P) / P;
          v.z = (float)cos(a1);
          v.w = (float)sin(a1);
        }
        coef[(size_t)k1 * kstride + (size_t)j * RQ + q] = v;
      }
    }
  }
  // launch geometry: nwr warps per row (GB coils each), several rows per CTA.  Small batches take
  // half as many rows per CTA, so the one-launch CG spreads a slice over twice as many CTAs
  // (measured on B300, 4 slices of 256 x 232 with 12 coils: 221 against 231 us per 10-iteration
  // solve; 16 slices keep two rows per tile: 782 against 1051 us with one).
  const int GB = 32 / Q;
  const int nwr = (pl->C + GB - 1) / GB;
  if (nwr > 8) return SENSE_OK;
  int rows = std::max(1, (pl->B <= 4 ? 4 : 8) / nwr);
  const int nwarps = rows * nwr;
  const NLLayout Lo = nl_layout(Q, P, J, kstride, rows, nwarps, GB, pl->S);
  if (Lo.total > 200 * 1024) return SENSE_OK;

  const size_t bc = coef.size() * sizeof(float4), bt = tw.size() * sizeof(float2);
  const size_t bw = wt.size() * sizeof(float), bs = sgn.size() * sizeof(float);
  const size_t bk = akx.size() * sizeof(int), bf = af.size() * sizeof(float);
  const size_t bl = std::max<size_t>(cols.size(), 1) * sizeof(int);
  char* d = nullptr;
  if (cudaMalloc(&d, bc + bt + bw + bs + bk + bf + bl + 64) != cudaSuccess) return SENSE_ECUDA;
  T.coef = reinterpret_cast<float4*>(d);
  T.tw = reinterpret_cast<float2*>(d + bc);
  T.wt = reinterpret_cast<float*>(d + bc + bt);
  T.sgn = reinterpret_cast<float*>(d + bc + bt + bw);
  T.akx = reinterpret_cast<int*>(d + bc + bt + bw + bs);
  T.af = reinterpret_cast<float*>(d + bc + bt + bw + bs + bk);
  T.cols = reinterpret_cast<int*>(d + bc + bt + bw + bs + bk + bf);
  T.ncols = (int)cols.size();
  if (cudaMemcpy(T.coef, coef.data(), bc, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.tw, tw.data(), bt, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.wt, wt.data(), bw, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.sgn, sgn.data(), bs, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.akx, akx.data(), bk, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.af, af.data(), bf, cudaMemcpyHostToDevice) != cudaSuccess ||
      (T.ncols > 0 && cudaMemcpy(T.cols, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                          cudaSuccess)) {
    cudaFree(d);
    T = LinesTables();
    return SENSE_ECUDA;
  }
  T.Q = Q; T.P = P; T.J = J; T.JMAX = JMAX; T.kstride = kstride;
  T.rows = rows; T.nwr = nwr; T.threads = nwarps * 32; T.smem = Lo.total;
  int maxb = 0;
  for (int mode = 0; mode < 4; ++mode) {
    NLKernel k = pick_kernel(Q, P, JMAX, mode, pl->S);
    if (!k) return SENSE_OK;  // no fused kernel for this (Q, P, sets): generic path
    int nb = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Lo.total) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, T.threads, Lo.total) != cudaSuccess)
      return SENSE_ECUDA;
    maxb = (mode == 0) ? nb : std::min(maxb, nb);
  }
  if (maxb < 1) return SENSE_OK;
  const int tiles = pl->B * ((pl->H + rows - 1) / rows);
  T.grid = std::min(tiles, maxb * pl->num_sms);
  T.ok = 1;
  // the whole-solve CG kernel: all of its CTAs must be resident at once (cooperative launch).
  // Used up to four tiles per CTA (measured on B300, 256x232, 12 coils, 10 iterations: 4 slices
  // 222 vs 360 us per solve, 16 slices with 3.5 tiles per CTA 0.93 vs 1.06 ms).
  if (pl->B <= kCoopMaxB) {
    CgKernel ck = Q == 8 ? pick_cg_q8(P, JMAX, pl->S) : pick_cg_q16(P, JMAX, pl->S);
    int nb = 0, coop = 0, dev = 0;
    if (ck && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, Lo.total) == cudaSuccess &&
        cudaFuncSetAttribute(ck, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ck, T.threads, Lo.total) == cudaSuccess && nb >= 1) {
      const int cgrid = std::min(tiles, nb * pl->num_sms);
      if (tiles <= 4 * cgrid) {
        T.coop = reinterpret_cast<const void*>(ck);
        T.coop_grid = cgrid;
      }
    }
  }
  return SENSE_OK;
}

void free_lines_tables(sense_plan pl) {
  if (pl->lines.coef) cudaFree(pl->lines.coef);
  pl->lines = LinesTables();
}

int launch_cg_lines(sense_plan pl, float2* x, int iters, double* rr_hist, const float2* rhs0, const double* lam,
                    int lam_count, const float2* rhs0b, float2* xlam) {
  const LinesTables& T = pl->lines;
  if (!T.coop) return SENSE_EUNSUPPORTED;
  Workspace& w = pl->w;
  NLArgs a;
  a.B = pl->B; a.C = pl->C; a.H = pl->H; a.HS = pl->S * pl->H; a.J = T.J; a.kstride = T.kstride;
  a.rows = T.rows; a.nwr = T.nwr;
  a.tiles_per_slice = (pl->H + T.rows - 1) / T.rows;
  a.ntiles = pl->B * a.tiles_per_slice;
  a.maps = pl->maps; a.coef = T.coef; a.tw = T.tw; a.wt = T.wt; a.sgn = T.sgn; a.akx = T.akx; a.af = T.af;
  a.x = w.r; a.pold = nullptr; a.pout = w.p; a.out = w.q; a.rhs = nullptr;
  a.lam_host = 0.f; a.lam_dev = lam; a.lam_shared = lam_count == 1;
  a.beta = nullptr; a.part = w.part; a.finalize = 0;
  a.rr = w.rr; a.alpha = w.alpha; a.rr_hist_row = nullptr;
  a.counter = w.counter; a.status = pl->status;
  CgCoop c;
  c.iters = iters; c.x = x; c.r = w.r; c.p = w.p; c.s = w.sv; c.w = w.wv; c.hist = rr_hist; c.rhs0 = rhs0;
  c.rhs0b = rhs0 ? rhs0b : nullptr; c.xlam = xlam;
  c.polls = pl->wait_polls; c.phantom = pl->wait_phantom;
  const size_t np = (size_t)pl->B * pl->S * pl->H;
  for (int i = 0; i < 2; ++i) {
    c.pd[i] = w.part2 + i * np;
    c.pg[i] = w.part2 + (2 + i) * np;
  }
  // counter block: last-block counter (bytes 0..127), scalars (512..895), and two sets of
  // per-slice arrival counts (set base + 128 b) and release words (set base + 2048 + 128 b) at
  // bytes 1024 and 5120.  Solves alternate between the sets; each zeroes the other set (the
  // previous solve's) after its wait for the previous kernel, so no reset sits in the stream
  // between the solve and the kernel before it (both sets are zero when the workspace is set up).
  c.sc = reinterpret_cast<double*>(w.counter + 128);
  const int set = pl->coop_set;
  pl->coop_set = 1 - set;
  c.cnt_s = w.counter + 256 + 1024 * set;
  c.rel_s = c.cnt_s + 512;
  c.cnt_o = w.counter + 256 + 1024 * (1 - set);
  void* args[] = {&a, &c};
  prof_mark("cg_lines", pl->stream, false);
  // cooperative launch with programmatic stream serialisation (the prologue overlaps the previous
  // kernel's tail); where the driver refuses the pair, the plain cooperative launch
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(T.coop_grid);
  cfg.blockDim = dim3(T.threads);
  cfg.dynamicSmemBytes = (size_t)T.smem;
  cfg.stream = pl->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelExC(&cfg, T.coop, args);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    e = cudaLaunchCooperativeKernel(T.coop, dim3(T.coop_grid), dim3(T.threads), args, (size_t)T.smem, pl->stream);
  }
  prof_mark("cg_lines", pl->stream, true);
  count_launch(pl);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}

int launch_normal_lines(sense_plan pl, const NormalLaunch& L) {
  const LinesTables& T = pl->lines;
  NLKernel k = pick_kernel(T.Q, T.P, T.JMAX, L.mode, pl->S);
  if (!k) return SENSE_EUNSUPPORTED;
  NLArgs a;
  a.B = pl->B; a.C = pl->C; a.H = pl->H; a.HS = pl->S * pl->H; a.J = T.J; a.kstride = T.kstride;
  a.rows = T.rows; a.nwr = T.nwr;
  a.tiles_per_slice = (pl->H + T.rows - 1) / T.rows;
  a.ntiles = pl->B * a.tiles_per_slice;
  a.maps = pl->maps; a.coef = T.coef; a.tw = T.tw; a.wt = T.wt; a.sgn = T.sgn; a.akx = T.akx; a.af = T.af;
  a.x = L.x; a.pold = L.pold; a.pout = L.pout; a.out = L.out; a.rhs = L.rhs;
  a.lam_host = L.lam_host; a.lam_dev = L.lam_dev;
  a.beta = L.beta; a.part = L.part; a.finalize = L.finalize;
  a.rr = pl->w.rr; a.alpha = pl->w.alpha; a.rr_hist_row = L.rr_hist_row;
  a.counter = pl->w.counter; a.status = pl->status;
  const char* group = L.mode == NM_ADJ ? "adjoint_lines" : "normal_lines";
  prof_mark(group, pl->stream, false);
  k<<<T.grid, T.threads, T.smem, pl->stream>>>(a);
  prof_mark(group, pl->stream, true);
  count_launch(pl);
  return cudaGetLastError() == cudaSuccess ? SENSE_OK : SENSE_ECUDA;
}
