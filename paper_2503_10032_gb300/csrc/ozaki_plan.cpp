// Plan of the tensor-core (BF16 slice) emulation of the setup GEMMs and the
// TMA tensor maps of the slice buffers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <unordered_map>

#include "ddelm_internal.h"

namespace ddelm {

namespace {
constexpr int OZ_BM = 128, OZ_BK = 64, OZ_KC = 1024;
// the all-levels shape: 128 x 48 tiles over 32-wide k blocks
constexpr int OZ_AL_BN = 48, OZ_AL_BK = 32;
// tile width of a phase: 128 (two levels per group) when every product has a
// contraction longer than one k-chunk, where A traffic dominates; else 64
// (four levels per group, combined exactly in integers)
constexpr int OZ_WIDE_K = 1024;
long long rup(long long x, long long a) { return (x + a - 1) / a * a; }
}  // namespace

int build_mixed(Plan &P, long long &cur) {
  auto take = [&](long long n) {
    long long off = cur;
    cur += (std::max(n, 1LL) + 31) / 32 * 32;
    return off;
  };
  // scale scratch: sized for the largest phase
  long long max_scales = 0;
  size_t max_slices = 0;
  const size_t n_setup = (size_t)P.ph_coarse;  // every wave's factorisation and local operator phases
  P.oz_phase.assign(P.setup_gemm.size(), OzPhase{0, 0, 0, 0, 0, 0, 0, 0, 64});
  struct Key {
    long long x;
    int ld, trans, R, K;
    bool operator==(const Key &o) const {
      return x == o.x && ld == o.ld && trans == o.trans && R == o.R && K == o.K;
    }
  };
  struct KeyHash {
    size_t operator()(const Key &k) const {
      unsigned long long h = (unsigned long long)k.x * 0x9E3779B97F4A7C15ull;
      h ^= ((unsigned long long)(unsigned)k.ld << 32 | (unsigned)k.R) + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
      h ^= ((unsigned long long)(unsigned)k.K << 1 | (unsigned)k.trans) + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
      return (size_t)h;
    }
  };
  // table sizes (upper bounds) up front: the plan is rebuilt on every setup
  {
    size_t nd = 0, nt = 0;
    for (size_t q = 0; q < (size_t)P.ph_coarse && q < P.setup_gemm.size(); ++q) {
      const GemmPhase &gp = P.setup_gemm[q];
      nd += gp.ndesc;
      for (int t = 0; t < gp.ndesc; ++t) {
        const GemmDesc &d = P.gdesc[gp.desc0 + t];
        nt += (size_t)((d.m + OZ_BM - 1) / OZ_BM) * ((d.n + 63) / 64);
      }
    }
    P.odesc.reserve(nd);
    P.sdesc.reserve(2 * nd);
    P.otile.reserve(3 * nt + 16);  // two tile lists, the 48-wide one up to 4/3 nt
  }
  std::vector<std::pair<int, long long>> scale_fix;  // (slice desc, relative scale offset)
  long long scale_base = 0;
  std::vector<int> phase_slices_begin;
  for (size_t q = 0; q < n_setup && q < P.setup_gemm.size(); ++q) {
    const GemmPhase &gp = P.setup_gemm[q];
    OzPhase op{int(P.sdesc.size()), 0, int(P.odesc.size()), 0, int(P.otile.size()), 0, 0, 0, 64, 0, 0, 64, 0, 0.0,
               0.0, 0ull};
    if (gp.ndesc == 0) {
      P.oz_phase[q] = op;
      continue;
    }
    const int S = q < P.setup_levels.size() ? P.setup_levels[q] : 9;  // 6 bits per level
    if (S < 1 || S > 10) {  // the fixed-point split holds 64^S in an int64
      P.err = "internal: slice level count";
      return DDELM_ERR_INVALID_ARG;
    }
    bool wide = gp.ndesc > 0, long_k = false;
    for (int t = 0; t < gp.ndesc; ++t) {
      wide = wide && P.gdesc[gp.desc0 + t].k > OZ_WIDE_K;
      long_k = long_k || P.gdesc[gp.desc0 + t].k > 16 * OZ_KC;
    }
    // the 96-bit integer sum of the four-level tiles holds up to 16 k-chunks
    // (|X| < 2^(43 + 48 + 4)); longer contractions take the FP64 combination
    wide = wide || long_k;
    // the rule: the all-levels shape (48 wide) unless the options ask for the
    // level-group shapes only or the contraction needs the FP64 combination;
    // the autotuner may switch to the alternative (the level-group rule's
    // width, or with tc_tiles = 1 the other level-group width; tc_tiles = 3
    // keeps the 64-wide level-group shape alone)
    const int grp_bn = (long_k || (wide && P.tc_tiles != 3)) ? 128 : 64;
    const int OZ_BN = (P.tc_tiles != 1 && P.tc_tiles != 3 && !long_k) ? OZ_AL_BN : grp_bn;
    std::unordered_map<Key, int, KeyHash> seen;
    seen.reserve(2 * (size_t)gp.ndesc);
    long long elem = 0, scl = 0;
    auto slice_of = [&](long long x, int ld, int trans, int R, int K) {
      Key k{x, ld, trans, R, K};
      auto it = seen.find(k);
      if (it != seen.end()) return it->second;
      SliceDesc s;
      std::memset(&s, 0, sizeof(s));
      s.x = x;
      s.ld = ld;
      s.trans = trans;
      s.R = R;
      s.K = K;
      s.Rpad = int(rup(R, OZ_BM));
      s.Kpad = int(rup(K, OZ_BK));
      s.S = S;
      s.out = elem;
      elem += (long long)S * s.Rpad * s.Kpad;
      // algorithmic bytes of the slicing: the source read twice (scale, digits), the slices written
      P.slice_bytes += 16.0 * R * (double)K + 2.0 * S * R * (double)rup(K, 8);
      s.scale = scl;  // relative; fixed below
      scl += rup(R, 32);
      int idx = int(P.sdesc.size());
      P.sdesc.push_back(s);
      seen[k] = idx;
      op.max_rpad = std::max(op.max_rpad, s.Rpad);
      op.max_kpad = std::max(op.max_kpad, s.Kpad);
      return idx;
    };
    op.overwrite = 1;
    for (int t = 0; t < gp.ndesc; ++t) {
      const GemmDesc &d = P.gdesc[gp.desc0 + t];
      if (d.beta != 0.0) op.overwrite = 0;
      const int sa = slice_of(d.a, d.lda, d.ta, d.m, d.k);
      const int sb = slice_of(d.b, d.ldb, d.tb ? 0 : 1, d.n, d.k);
      OzDesc o;
      std::memset(&o, 0, sizeof(o));
      o.c = d.c;
      o.m = d.m;
      o.n = d.n;
      o.ldc = d.ldc;
      o.S = S;
      o.kc = OZ_KC;
      o.Kpad = int(rup(d.k, OZ_BK));
      o.RpadA = P.sdesc[sa].Rpad;
      o.RpadB = P.sdesc[sb].Rpad;
      o.tmapA = sa;
      o.tmapB = sb;
      o.scaleA = P.sdesc[sa].scale;  // relative for now
      o.scaleB = P.sdesc[sb].scale;
      o.alpha = d.alpha;
      o.beta = d.beta;
      P.odesc.push_back(o);
      op.ndesc++;
    }
    // tile lists: the rule's width, then (for the autotuner) the other one
    double pairs = 0;  // tensor-core work: every level's pairs over the k blocks a tile needs
    for (int l = 0; l < S; ++l) pairs += l + 1;
    // k blocks are 64 wide for the level-group shapes, 32 for the all-levels one
    auto emit_tiles = [&](int BN, int &ntile, double &flops) {
      const int BK = BN == OZ_AL_BN ? OZ_AL_BK : OZ_BK;
      for (int t = 0; t < gp.ndesc; ++t) {
        const GemmDesc &d = P.gdesc[gp.desc0 + t];
        const int di = op.desc0 + t;
        const int tm = (d.m + OZ_BM - 1) / OZ_BM, tn = (d.n + BN - 1) / BN;
        const int nkb = (d.k + BK - 1) / BK;  // blocks wholly past k would load only zeros
        for (int x = 0; x < tm; ++x)
          for (int y = 0; y < tn; ++y) {
            if (d.syrk && x * OZ_BM >= (y + 1) * BN) continue;  // strictly below the diagonal
            int kb0 = 0, kb1 = nkb;
            // op(B)[k][j] = 0 for k > j ; op(A)[i][k] = 0 for k < i
            if (d.flags & GEMM_B_UPPER) kb1 = std::min(kb1, ((y + 1) * BN + BK - 1) / BK);
            if (d.flags & GEMM_A_UPPER) kb0 = std::max(kb0, x * (OZ_BM / BK));
            if (kb1 < kb0) kb1 = kb0;
            P.otile.push_back({di, x, y, kb0, kb1, 0, 0, 0});
            ntile++;
            flops += 2.0 * OZ_BM * BN * (double)(kb1 - kb0) * BK * pairs;
          }
      }
    };
    // the autotuner's key: the phase's product shapes and tile options
    {
      unsigned long long k = 1469598103934665603ull;  // FNV-1a
      auto mix = [&](long long v) {
        for (int b = 0; b < 8; ++b) {
          k ^= (unsigned long long)((v >> (8 * b)) & 0xff);
          k *= 1099511628211ull;
        }
      };
      mix(P.tc_tiles);
      mix(S);
      mix(gp.ndesc);
      for (int t = 0; t < gp.ndesc; ++t) {
        const GemmDesc &d = P.gdesc[gp.desc0 + t];
        mix(d.m);
        mix(d.n);
        mix(d.k);
        mix(d.flags | (d.syrk ? 1 << 20 : 0));
      }
      op.key = k;
    }
    int bn_rule = OZ_BN, bn_alt = OZ_BN == OZ_AL_BN ? grp_bn : (OZ_BN == 64 ? 128 : 64);
    bool with_alt = P.autotune && op.overwrite && !long_k && P.tc_tiles < 2;
    if (with_alt) {
      // a width chosen for this shape by an earlier handle's autotuner: that
      // list alone (nothing left to time)
      const int known = tuned_tile_width(op.key);
      if (known == bn_alt) std::swap(bn_rule, bn_alt);
      if (known == bn_rule) {
        with_alt = false;
        P.tune_from_cache++;
      }
    }
    op.bn = bn_rule;
    emit_tiles(bn_rule, op.ntile, op.flops);
    P.oz_flops += op.flops;
    op.bn_alt = bn_alt;
    op.tile0_alt = int(P.otile.size());
    if (with_alt) emit_tiles(op.bn_alt, op.ntile_alt, op.flops_alt);
    for (const int bn : {op.bn, op.ntile_alt > 0 ? op.bn_alt : op.bn}) {
      if (bn == OZ_AL_BN) P.maps_al = true;
      else P.maps_grp = true;
    }
    op.nslice = int(P.sdesc.size()) - op.slice0;
    for (int t = op.slice0; t < op.slice0 + op.nslice; ++t)
      if (P.sdesc[t].S != S) {  // the slicing launch takes one level count
        P.err = "internal: slice levels within a phase";
        return DDELM_ERR_INVALID_ARG;
      }
    P.oz_phase[q] = op;
    max_scales = std::max(max_scales, scl);
    max_slices = std::max(max_slices, (size_t)elem * 2);
  }
  scale_base = take(max_scales);
  for (auto &s : P.sdesc) s.scale += scale_base;
  for (auto &o : P.odesc) {
    o.scaleA += scale_base;
    o.scaleB += scale_base;
  }
  P.bytes_slices = rup((long long)max_slices, 1024);
  return DDELM_OK;
}

// Three 3-D tensor maps per slice buffer i, each over S levels of R rows of K
// BF16 (row stride Kpad, level stride Rpad Kpad): map i with box 64 x 64 x 1
// and the 128-byte swizzle (the level-group shapes), maps n + 2 i and
// n + 2 i + 1 (n slice buffers) with boxes 32 x 128 x S and 32 x 48 x S and
// the 64-byte swizzle (the all-levels shape's A and B sides); all are the
// canonical K-major layouts tcgen05 reads.  Boxes reaching past R or K are
// zero-filled by the copy, so the slicing writes no padding.
int encode_tensor_maps(const Plan &P, void *ws, std::vector<unsigned char> &maps) {
  maps.assign(std::max<size_t>(P.sdesc.size(), 1) * 3 * 128, 0);
  if (P.sdesc.empty()) return DDELM_OK;
  typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                               const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return DDELM_ERR_CUDA;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  char *slices = static_cast<char *>(ws) + P.off_slices;
  for (size_t i = 0; i < P.sdesc.size(); ++i) {
    const SliceDesc &s = P.sdesc[i];
    void *gaddr = slices + s.out * 2;
    if ((reinterpret_cast<uintptr_t>(gaddr) & 15u) != 0) return DDELM_ERR_INVALID_ARG;
    cuuint64_t dims[3] = {(cuuint64_t)s.K, (cuuint64_t)s.R, (cuuint64_t)s.S};
    cuuint64_t strides[2] = {(cuuint64_t)s.Kpad * 2, (cuuint64_t)s.Rpad * (cuuint64_t)s.Kpad * 2};
    cuuint32_t estr[3] = {1, 1, 1};
    const size_t slot[3] = {i, P.sdesc.size() + 2 * i, P.sdesc.size() + 2 * i + 1};
    const cuuint32_t boxes[3][3] = {{64, 64, 1},
                                    {(cuuint32_t)OZ_AL_BK, (cuuint32_t)OZ_BM, (cuuint32_t)s.S},
                                    {(cuuint32_t)OZ_AL_BK, (cuuint32_t)OZ_AL_BN, (cuuint32_t)s.S}};
    for (int v = 0; v < 3; ++v) {
      if (v == 0 ? !P.maps_grp : !P.maps_al) continue;  // no tile list reads through this family
      CUtensorMap m;
      CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, gaddr, dims, strides, boxes[v], estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, v == 0 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return DDELM_ERR_CUDA;
      std::memcpy(maps.data() + slot[v] * 128, &m, 128);
    }
  }
  return DDELM_OK;
}

}  // namespace ddelm
