// One local ridge least-squares solve, C = K^+ F, that allocates no device
// memory: its scratch is a file-scope static device array, for callers that
// cannot call cudaMalloc (for example code running where the allocator is off
// limits, or hosts that hand this library only fixed, pre-registered memory).
// The arithmetic is the library's own: shifted CholeskyQR3 of [K; eps I] on
// the FP64 GEMM and Cholesky kernels.  The paper has no counterpart.
#include <cstring>
#include <mutex>
#include <vector>

#include "ddelm_internal.h"

namespace {

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) double g_static_scratch[DDELM_STATIC_SCRATCH_DOUBLES];

std::mutex g_mu;
double *g_addr[256] = {};

// Device address of the array for the current device (the host-side symbol
// is only a stand-in).  Resolved once per device, with that device current.
int scratch_base(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DDELM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return DDELM_ERR_CUDA;
    g_addr[dev] = static_cast<double *>(p);
  }
  *out = g_addr[dev];
  return DDELM_OK;
}

long long rup32(long long n) { return (n + 31) / 32 * 32; }

}  // namespace

using namespace ddelm;

extern "C" int ddelm_local_lstsq_static(const double *d_K, int m, int M, const double *d_F, int R,
                                        double eps_rel, double *d_C, void *stream) {
  if (!d_K || !d_F || !d_C || m < 1 || M < 1 || M > 256 || R < 1 || R > 16 || !(eps_rel >= 0.0)) {
    record_plan_error("ddelm_local_lstsq_static: null pointer, or m < 1, M outside 1..256, R outside 1..16, "
                      "eps_rel < 0");
    return DDELM_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The tables (GEMM descriptors and tiles, Cholesky descriptors) come first in
  // the array; their size depends on m and M, so they are built before the
  // data regions are laid out behind them.  Data offsets are fixed here as
  // offsets from the end of the tables (DB0, known once the tables are built).
  long long cur = 0;
  auto take = [&](long long n) {
    long long o = cur;
    cur += rup32(n);
    return o;
  };
  // layout (doubles): K copy (later Q2) | F | Q1 | G V1 V2 V3 Z1 Z2 T1 V | T Qtf C | status
  const long long oK = take((long long)m * M), oF = take((long long)m * R), oQ1 = take((long long)m * M);
  const long long oG = take((long long)M * M), oV1 = take((long long)M * M), oV2 = take((long long)M * M);
  const long long oV3 = take((long long)M * M), oZ1 = take((long long)M * M), oZ2 = take((long long)M * M);
  const long long oT1 = take((long long)M * M), oV = take((long long)M * M);
  const long long oT = take((long long)M * R), oQtf = take((long long)M * R), oC = take((long long)M * R);
  const long long oSt = take(64);
  const long long data_doubles = cur;
  if (data_doubles > DDELM_STATIC_SCRATCH_DOUBLES) {
    record_plan_error("ddelm_local_lstsq_static: the sizes need more scratch than the static array holds");
    return DDELM_ERR_INVALID_ARG;
  }

  // tables: one phase per dependent step; descriptor offsets are relative to
  // the start of the data regions and shifted once DB0 is known
  std::vector<GemmDesc> gd;
  std::vector<GemmTile> gt;
  struct Ph {
    int t0, nt, skinny;
  };
  std::vector<Ph> phases;
  auto begin = [&](int skinny) { phases.push_back({int(gt.size()), 0, skinny}); };
  auto add = [&](long long a, long long b, long long c, int mm, int nn, int kk, int lda, int ldb, int ldc, int ta,
                 int tb, int flags, double alpha, double beta, bool upper) {
    GemmDesc d;
    std::memset(&d, 0, sizeof(d));
    d.a = a;
    d.b = b;
    d.c = c;
    d.m = mm;
    d.n = nn;
    d.k = kk;
    d.lda = lda;
    d.ldb = ldb;
    d.ldc = ldc;
    d.ta = ta;
    d.tb = tb;
    d.flags = flags;
    d.syrk = upper ? 1 : 0;
    d.alpha = alpha;
    d.beta = beta;
    const int di = int(gd.size());
    gd.push_back(d);
    Ph &ph = phases.back();
    if (ph.skinny) {
      for (int x = 0; x < (mm + 31) / 32; ++x) gt.push_back({di, x, 0, 0}), ph.nt++;
      return;
    }
    for (int x = 0; x < (mm + 63) / 64; ++x)
      for (int y = 0; y < (nn + 63) / 64; ++y) {
        if (upper && x > y) continue;
        gt.push_back({di, x, y, 0});
        ph.nt++;
      }
  };
  const int BU = GEMM_B_UPPER, AU = GEMM_A_UPPER;
  begin(0);  // 0: G = K^T K
  add(oK, oK, oG, M, M, m, M, M, M, 1, 0, 0, 1.0, 0.0, true);
  begin(0);  // 1: Q1 = K V1
  add(oK, oV1, oQ1, m, M, M, M, M, M, 0, 0, BU, 1.0, 0.0, false);
  begin(0);  // 2: G = Q1^T Q1
  add(oQ1, oQ1, oG, M, M, m, M, M, M, 1, 0, 0, 1.0, 0.0, true);
  begin(0);  // 3: G += Z1^T Z1
  add(oZ1, oZ1, oG, M, M, M, M, M, M, 1, 0, BU, 1.0, 1.0, true);
  begin(0);  // 4: Q2 = Q1 V2 (over the K copy), Z2 = Z1 V2
  add(oQ1, oV2, oK, m, M, M, M, M, M, 0, 0, BU, 1.0, 0.0, false);
  add(oZ1, oV2, oZ2, M, M, M, M, M, M, 0, 0, BU | AU, 1.0, 0.0, false);
  begin(0);  // 5: G = Q2^T Q2
  add(oK, oK, oG, M, M, m, M, M, M, 1, 0, 0, 1.0, 0.0, true);
  begin(0);  // 6: G += Z2^T Z2
  add(oZ2, oZ2, oG, M, M, M, M, M, M, 1, 0, BU, 1.0, 1.0, true);
  begin(0);  // 7: T1 = V1 V2
  add(oV1, oV2, oT1, M, M, M, M, M, M, 0, 0, AU | BU, 1.0, 0.0, false);
  begin(0);  // 8: V = T1 V3
  add(oT1, oV3, oV, M, M, M, M, M, M, 0, 0, AU | BU, 1.0, 0.0, false);
  begin(1);  // 9: T = Q2^T F
  add(oK, oF, oT, M, R, m, M, R, R, 1, 0, 0, 1.0, 0.0, false);
  begin(1);  // 10: Qtf = V3^T T
  add(oV3, oT, oQtf, M, R, M, M, R, R, 1, 0, 0, 1.0, 0.0, false);
  begin(1);  // 11: C = V Qtf
  add(oV, oQtf, oC, M, R, M, M, R, R, 0, 0, AU, 1.0, 0.0, false);
  std::vector<CholDesc> cd(3);
  const double u = 1.1102230246251565e-16;
  for (int k = 0; k < 3; ++k) {
    std::memset(&cd[k], 0, sizeof(CholDesc));
    cd[k].g = oG;
    cd[k].v = k == 0 ? oV1 : k == 1 ? oV2 : oV3;
    cd[k].z = k == 0 ? oZ1 : -1;
    cd[k].M = M;
    cd[k].m = m;
    cd[k].w = -1;
    cd[k].epsout = -1;
    cd[k].ridge = k == 0;
    cd[k].shift_kind = k == 0 ? 1 : 0;
    cd[k].status = k;
    cd[k].eps_rel = eps_rel;
    cd[k].shift_rel = 11.0 * (double(m + M) * M + double(M) * (M + 1)) * u;
  }
  const size_t bytes_gd = gd.size() * sizeof(GemmDesc), bytes_gt = gt.size() * sizeof(GemmTile);
  const size_t off_gt = (bytes_gd + 255) / 256 * 256, off_cd = off_gt + (bytes_gt + 255) / 256 * 256;
  const size_t bytes_tab = off_cd + cd.size() * sizeof(CholDesc);
  const long long DB0 = rup32((long long)((bytes_tab + sizeof(double) - 1) / sizeof(double)));
  if (DB0 + data_doubles > DDELM_STATIC_SCRATCH_DOUBLES) {
    record_plan_error("ddelm_local_lstsq_static: the sizes need more scratch (tables and data) than the static "
                      "array holds");
    return DDELM_ERR_INVALID_ARG;
  }
  for (auto &d : gd) {
    d.a += DB0;
    d.b += DB0;
    d.c += DB0;
  }
  for (auto &c : cd) {
    c.g += DB0;
    c.v += DB0;
    if (c.z >= 0) c.z += DB0;
  }
  std::vector<char> tab(bytes_tab, 0);
  std::memcpy(tab.data(), gd.data(), bytes_gd);
  std::memcpy(tab.data() + off_gt, gt.data(), bytes_gt);
  std::memcpy(tab.data() + off_cd, cd.data(), cd.size() * sizeof(CholDesc));

  double *db = nullptr;
  int rc = scratch_base(&db);
  if (rc != DDELM_OK) return rc;
#define CKS(x)                                         \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) {                           \
      record_cuda_error(e_, #x, __FILE__, __LINE__);   \
      return DDELM_ERR_CUDA;                           \
    }                                                  \
  } while (0)
  char *base = reinterpret_cast<char *>(db);
  // the host table is pageable: cudaMemcpyAsync has consumed it when it returns
  CKS(cudaMemcpyAsync(base, tab.data(), bytes_tab, cudaMemcpyHostToDevice, s));
  CKS(cudaMemcpyAsync(db + DB0 + oK, d_K, sizeof(double) * (size_t)m * M, cudaMemcpyDeviceToDevice, s));
  CKS(cudaMemcpyAsync(db + DB0 + oF, d_F, sizeof(double) * (size_t)m * R, cudaMemcpyDeviceToDevice, s));
  CKS(cudaMemsetAsync(db + DB0 + oSt, 0, 64 * sizeof(double), s));  // status words start at zero
  const GemmDesc *dgd = reinterpret_cast<const GemmDesc *>(base);
  const GemmTile *dgt = reinterpret_cast<const GemmTile *>(base + off_gt);
  const CholDesc *dcd = reinterpret_cast<const CholDesc *>(base + off_cd);
  int *status = reinterpret_cast<int *>(db + DB0 + oSt);
  auto gemm = [&](int k) {
    return launch_gemm_table(dgd, dgt + phases[k].t0, phases[k].nt, db, phases[k].skinny, s);
  };
  CKS(gemm(0));
  CKS(launch_chol_table(dcd + 0, 1, M, db, status, s));
  CKS(gemm(1));
  CKS(gemm(2));
  CKS(gemm(3));
  CKS(launch_chol_table(dcd + 1, 1, M, db, status, s));
  CKS(gemm(4));
  CKS(gemm(5));
  CKS(gemm(6));
  CKS(launch_chol_table(dcd + 2, 1, M, db, status, s));
  for (int k = 7; k <= 11; ++k) CKS(gemm(k));
  CKS(cudaMemcpyAsync(d_C, db + DB0 + oC, sizeof(double) * (size_t)M * R, cudaMemcpyDeviceToDevice, s));
  int st[3] = {0, 0, 0};
  CKS(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
#undef CKS
  return (st[0] || st[1] || st[2]) ? DDELM_ERR_RANK_DEFICIENT : DDELM_OK;
}
