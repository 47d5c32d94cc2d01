/*
 * CPU oracle for the variance-adaptive multi-resolution TSDF map (MrHash, arXiv 2511.21459).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the CUDA library is checked against. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it. It shares no code, header or table with
 * the CUDA library.
 *
 * What it computes, step by step, per frame (paper section in brackets):
 *   rays                    camera: pixel ray and range; LiDAR: sensor origin to point       [Sec. 3.1, Eq. 1/2]
 *   allocation              every voxel block whose cell meets the ray's truncation band      [Sec. 3.2, DDA]
 *   fusion                  truncated signed distance per voxel, running mean and weight     [Eq. 1, Eq. 2, Eq. 3]
 *   Welford variance        S2 += (d - D_old)(d - D_new), sigma^2 = S2 / k                   [Sec. 3.2.1, Eq. 5/6]
 *   block variance          mean of voxel variances over observed voxels of a block          [Sec. 3.2.1]
 *   re-levelling            low-variance block -> coarser level (merge); high-variance block [Sec. 3.2.1, Fig. 2/4]
 *                           -> finer level (split, an extension with hysteresis)
 *   raycast                 first zero crossing of the trilinear field along each pixel ray  [Fig. 2 "render"]
 * The readings taken where the paper is silent are written next to the code that takes them.
 *
 * Two arithmetic modes:
 *   f64  - all voxel arithmetic and storage in double: the accuracy truth.
 *   f32s - float storage and float arithmetic in the literal operation order written below. Compile with
 *          -ffp-contract=off so no multiply-add is fused. Optional half storage of D and colour.
 * Block keys are decided by exact integer arithmetic on fixed-point segment endpoints in both modes, so the key set
 * does not depend on the mode.
 *
 * Plain containers only: std::unordered_map from block key to block, std::vector voxel arrays.
 */
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

// ------------------------------------------------------------------------------------------------ constants

constexpr int kFineDim = 8;           // voxels per block side at the finest level (512-voxel blocks, Sec. 4.1.4)
constexpr int kFracBits = 16;         // fixed-point fraction bits per block edge for segment endpoints
constexpr int64_t kBlockUnit = int64_t(1) << kFracBits;
constexpr int64_t kVoxelUnit = kBlockUnit / kFineDim;  // one finest voxel
constexpr int64_t kKeyLimit = (int64_t(1) << 20) - 2;  // |block coordinate| bound (21-bit packed keys)
constexpr int kMaxLevels = 3;

struct Key {
  int64_t x, y, z;
  bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
  bool operator<(const Key& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ULL;
    h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4FULL + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.z * 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// ---------------------------------------------------------------------------------------- exact segment geometry
//
// Allocation (Sec. 3.2, "leverage DDA ... to allocate all intersected voxel blocks") needs the set of cells a segment
// meets. Cells are half-open [c U, (c+1) U)^3. Endpoints are fixed-point integers, so "the closed segment meets the
// cell" is decided exactly with integer arithmetic.

struct Frac {  // num / den with den > 0, plus whether the bound is attained
  __int128 num, den;
  bool closed;
};

int frac_cmp(const Frac& a, const Frac& b) {
  __int128 l = a.num * b.den, r = b.num * a.den;
  return l < r ? -1 : (l > r ? 1 : 0);
}

// True iff the closed segment A -> B meets the half-open cell [c U, (c+1) U)^3.
bool segment_meets_cell(const int64_t A[3], const int64_t B[3], const int64_t c[3], int64_t U) {
  Frac lo{0, 1, true}, hi{1, 1, true};
  for (int i = 0; i < 3; ++i) {
    int64_t d = B[i] - A[i];
    int64_t L = c[i] * U, H = (c[i] + 1) * U;
    if (d == 0) {
      if (A[i] < L || A[i] >= H) return false;
      continue;
    }
    Frac cand_lo, cand_hi;
    if (d > 0) {  // A + s d >= L  <=>  s >= (L - A)/d ;  A + s d < H  <=>  s < (H - A)/d
      cand_lo = Frac{(__int128)(L - A[i]), (__int128)d, true};
      cand_hi = Frac{(__int128)(H - A[i]), (__int128)d, false};
    } else {      // A + s d >= L  <=>  s <= (A - L)/|d| ;  A + s d < H  <=>  s > (A - H)/|d|
      cand_hi = Frac{(__int128)(A[i] - L), (__int128)(-d), true};
      cand_lo = Frac{(__int128)(A[i] - H), (__int128)(-d), false};
    }
    int cl = frac_cmp(cand_lo, lo);
    if (cl > 0 || (cl == 0 && !cand_lo.closed)) lo = cand_lo;
    int ch = frac_cmp(cand_hi, hi);
    if (ch < 0 || (ch == 0 && !cand_hi.closed)) hi = cand_hi;
  }
  int cmp = frac_cmp(lo, hi);
  return cmp < 0 || (cmp == 0 && lo.closed && hi.closed);
}

// Every cell (edge U) the closed segment A -> B meets, by testing each cell of the bounding box.
std::vector<Key> cells_bruteforce(const int64_t A[3], const int64_t B[3], int64_t U) {
  int64_t lo[3], hi[3];
  for (int i = 0; i < 3; ++i) {
    int64_t a = floor_div(A[i], U), b = floor_div(B[i], U);
    lo[i] = std::min(a, b);
    hi[i] = std::max(a, b);
  }
  std::vector<Key> out;
  for (int64_t x = lo[0]; x <= hi[0]; ++x)
    for (int64_t y = lo[1]; y <= hi[1]; ++y)
      for (int64_t z = lo[2]; z <= hi[2]; ++z) {
        int64_t c[3] = {x, y, z};
        if (segment_meets_cell(A, B, c, U)) out.push_back(Key{x, y, z});
      }
  return out;
}

// The same cells in the order the segment visits them: an Amanatides-Woo walk whose boundary crossings are compared
// exactly. Crossing a boundary upward enters the next cell at the crossing point itself; crossing downward enters it
// just after (cells are half-open). When crossings coincide, the upward ones are taken together first, then the
// downward ones together.
std::vector<Key> cells_dda(const int64_t A[3], const int64_t B[3], int64_t U) {
  int64_t cell[3], end[3], D[3], N[3];
  for (int i = 0; i < 3; ++i) {
    cell[i] = floor_div(A[i], U);
    end[i] = floor_div(B[i], U);
    D[i] = B[i] - A[i];
    // distance along axis i from A to the next boundary crossing (always >= 0)
    if (D[i] > 0) N[i] = (cell[i] + 1) * U - A[i];
    else if (D[i] < 0) N[i] = A[i] - cell[i] * U;
    else N[i] = 0;
  }
  std::vector<Key> out;
  out.push_back(Key{cell[0], cell[1], cell[2]});
  for (int guard = 0; guard < 1 << 20; ++guard) {
    if (cell[0] == end[0] && cell[1] == end[1] && cell[2] == end[2]) break;
    // smallest crossing parameter N_i / |D_i| among moving axes
    int best = -1;
    for (int i = 0; i < 3; ++i) {
      if (D[i] == 0) continue;
      if (best < 0) { best = i; continue; }
      __int128 l = (__int128)N[i] * (D[best] < 0 ? -D[best] : D[best]);
      __int128 r = (__int128)N[best] * (D[i] < 0 ? -D[i] : D[i]);
      if (l < r) best = i;
    }
    bool tie[3] = {false, false, false};
    for (int i = 0; i < 3; ++i) {
      if (D[i] == 0) continue;
      __int128 l = (__int128)N[i] * (D[best] < 0 ? -D[best] : D[best]);
      __int128 r = (__int128)N[best] * (D[i] < 0 ? -D[i] : D[i]);
      tie[i] = (l == r);
    }
    bool any_up = false, any_down = false;
    for (int i = 0; i < 3; ++i) {
      if (!tie[i]) continue;
      if (D[i] > 0) any_up = true; else any_down = true;
    }
    if (any_up) {
      for (int i = 0; i < 3; ++i)
        if (tie[i] && D[i] > 0) { cell[i] += 1; N[i] += U; }
      out.push_back(Key{cell[0], cell[1], cell[2]});
    }
    if (any_down) {
      if (cell[0] == end[0] && cell[1] == end[1] && cell[2] == end[2]) break;
      for (int i = 0; i < 3; ++i)
        if (tie[i] && D[i] < 0) { cell[i] -= 1; N[i] += U; }
      out.push_back(Key{cell[0], cell[1], cell[2]});
    }
  }
  return out;
}

bool key_in_range(const Key& k) {
  return k.x >= -kKeyLimit && k.x <= kKeyLimit && k.y >= -kKeyLimit && k.y <= kKeyLimit && k.z >= -kKeyLimit &&
         k.z <= kKeyLimit;
}

// float -> fixed point: floor(x * S), only for |x * S| < 2^40 (otherwise the ray is dropped)
bool to_fixed_f(float v, float S, int64_t* out) {
  float p = v * S;
  if (!(std::fabs(p) < 1099511627776.0f)) return false;
  *out = (int64_t)std::floor(p);
  return true;
}
bool to_fixed_d(double v, double S, int64_t* out) {
  double p = v * S;
  if (!(std::fabs(p) < 1099511627776.0)) return false;
  *out = (int64_t)std::floor(p);
  return true;
}

// ------------------------------------------------------------------------------------------------ half storage

float half_round(float x) { return (float)(_Float16)x; }

template <class S> struct Store;
template <> struct Store<double> {
  static double put(double x) { return x; }
  static double get(double x) { return x; }
};
template <> struct Store<float> {
  static float put(float x) { return x; }
  static float get(float x) { return x; }
};
template <> struct Store<_Float16> {
  static _Float16 put(float x) { return (_Float16)x; }
  static float get(_Float16 x) { return (float)x; }
};

}  // namespace

// ------------------------------------------------------------------------------------------------ C interface types

extern "C" {

struct orc_params {
  float base_voxel;        // coarsest-level voxel edge [m]
  int n_levels;            // 1..3
  float truncation;        // tau [m]
  double var_threshold[2]; // theta_l: merge l -> l+1 when the block variance is below it [m^2]
  double split_hysteresis; // h: split l -> l-1 when the block variance exceeds h * theta_{l-1}; 0 disables
  int min_obs;             // k_min: mean weight over observed voxels needed before a block may change level
  int precision;           // 0 = f32s, 1 = f64
  int fp16;                // f32s only: D and colour stored as half
  int has_color;
  float min_range, max_range;  // LiDAR validity of |x_s| [m]
};

struct orc_pinhole {
  float fx, fy, cx, cy;
  int width, height;
  float min_depth, max_depth;
};

struct orc_frame_stats {
  int64_t valid_rays, touched, new_blocks, merged, split, fp64_rechecks, observations;
  int64_t updated_voxels;  // distinct voxels updated by the frame
  int64_t evicted, restored;  // streaming: blocks moved to the archive before the frame, and back by it
};

// learned level predictor (level_predictor.cpp)
int orc_block_features(const orc_pinhole* K, const float* R, const float* t, const float* rho, float E, float tau,
                       int64_t bx, int64_t by, int64_t bz, const uint16_t* w, int n_levels, float* f, int* level);
void orc_lidar_block_features(const uint64_t* mom, const double* T_ws, float E, float tau, int64_t bx, int64_t by,
                              int64_t bz, const uint16_t* w, int n_levels, float* f, int* level);

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------------------ the map

template <class R, class Sto>
struct Block {
  int level = 0;
  std::vector<Sto> D;
  std::vector<R> W, S2;
  std::vector<Sto> C[3];
  void resize(int n, bool color) {
    size_t v = (size_t)n * n * n;
    D.assign(v, Store<Sto>::put(0));
    W.assign(v, 0);
    S2.assign(v, 0);
    for (int c = 0; c < 3; ++c) C[c].assign(color ? v : 0, Store<Sto>::put(0));
  }
};

struct MapBase {
  virtual ~MapBase() {}
  virtual int integrate_depth(const orc_pinhole*, const double*, const float*, const uint8_t*, orc_frame_stats*) = 0;
  virtual int integrate_points(const double*, const float*, int64_t, orc_frame_stats*) = 0;
  virtual int raycast(const orc_pinhole*, const double*, float*, float*, uint8_t*) = 0;
  virtual int raycast_pixels(const orc_pinhole*, const double*, int64_t, const int64_t*, float*, float*,
                             uint8_t*) const = 0;
  virtual void probe_points(int64_t, const double*, double*, int8_t*, float*, uint8_t*) const = 0;
  virtual int set_block(const int32_t*, int, const double*, const double*, const double*, const double*) = 0;
  virtual void extract_mesh(std::vector<float>& tris) const = 0;
  virtual void set_streaming(float fraction, float radius, const int64_t* max_blocks) = 0;
  virtual int64_t archived() const = 0;
  std::vector<float> mesh;  // last extracted triangle soup
  virtual int64_t count_blocks(int64_t* n_voxels) = 0;
  virtual int extract(int32_t*, uint8_t*, int64_t*, double*, double*, double*, double*) = 0;
  virtual int block_stats(int32_t*, uint8_t*, double*, int64_t*, int64_t*) = 0;
  virtual int resample(int, int, const double*, const double*, const double*, const double*, double*, double*,
                       double*, double*) = 0;
  // learned level predictor (camera frames): BF16 weights, or empty for the plain rule
  std::vector<uint16_t> pred_w;
  // feature records of new blocks (training data), when capture is on
  bool capture = false;
  std::vector<Key> cap_keys;
  std::vector<float> cap_feat;
};

// ---- Marching Cubes case table (Lorensen and Cline's cube cases), built here from its definition rather than copied.
// Corner c of a cell has offset (c & 1, (c >> 1) & 1, (c >> 2) & 1); a corner is inside when its value is below zero.
// Edge 4a + r joins corner c0 and c0 | 1 << a, where c0 is the r-th corner (ascending) whose bit a is clear. On each
// face the corners are walked counter-clockwise as seen from outside the cell; the surface crosses an edge where the
// walk passes between an inside and an outside corner, and every crossing entering the inside is joined to the next
// crossing (in walk order) leaving it, so that two diagonal inside corners of a face stay separated. Joined across the
// six faces the segments close into loops, each fanned into triangles from its lowest edge; the triangles then face
// the outside (increasing value).
struct McTable {
  int n_tris[256];
  int8_t edges[256][36];
  int8_t edge_corner[12][2];
  McTable() {
    int e = 0;
    for (int a = 0; a < 3; ++a)
      for (int c0 = 0; c0 < 8; ++c0)
        if (!((c0 >> a) & 1)) {
          edge_corner[e][0] = (int8_t)c0;
          edge_corner[e][1] = (int8_t)(c0 | (1 << a));
          ++e;
        }
    auto edge_of = [&](int c0, int c1) {
      for (int k = 0; k < 12; ++k)
        if ((edge_corner[k][0] == c0 && edge_corner[k][1] == c1) || (edge_corner[k][0] == c1 && edge_corner[k][1] == c0))
          return k;
      return -1;
    };
    for (int cs = 0; cs < 256; ++cs) {
      int next[12];
      for (int k = 0; k < 12; ++k) next[k] = -1;
      for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
          const int u = (a + 1) % 3, w = (a + 2) % 3;
          static const int ccw[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
          int q[4];
          for (int i = 0; i < 4; ++i) {
            const int* uw = side ? ccw[i] : ccw[(4 - i) % 4];
            q[i] = (side << a) | (uw[0] << u) | (uw[1] << w);
          }
          int cross[4], enters[4], nc = 0;
          for (int i = 0; i < 4; ++i) {
            const int c0 = q[i], c1 = q[(i + 1) % 4];
            const int in0 = (cs >> c0) & 1, in1 = (cs >> c1) & 1;
            if (in0 != in1) {
              cross[nc] = edge_of(c0, c1);
              enters[nc] = in1;
              ++nc;
            }
          }
          for (int i = 0; i < nc; ++i)
            if (enters[i]) next[cross[i]] = cross[(i + 1) % nc];
        }
      int nt = 0;
      bool seen[12] = {false};
      for (int k = 0; k < 12; ++k) {
        if (next[k] < 0 || seen[k]) continue;
        int loop[12], len = 0, f = k;
        do {
          seen[f] = true;
          loop[len++] = f;
          f = next[f];
        } while (f != k);
        for (int i = 1; i + 1 < len; ++i) {
          edges[cs][3 * nt] = (int8_t)loop[0];
          edges[cs][3 * nt + 1] = (int8_t)loop[i];
          edges[cs][3 * nt + 2] = (int8_t)loop[i + 1];
          ++nt;
        }
      }
      n_tris[cs] = nt;
    }
  }
};

template <class R, class Sto>
struct Map : MapBase {
  orc_params P;
  int L;
  R tau;
  R v[kMaxLevels];        // voxel edge per level
  int n[kMaxLevels];      // voxels per block side per level
  float E_f;              // block edge (float), the unit of the fixed-point key coordinates
  std::unordered_map<Key, Block<R, Sto>, KeyHash> blocks;

  explicit Map(const orc_params& p) : P(p), L(p.n_levels) {
    tau = (R)p.truncation;
    float v0f = p.base_voxel / (float)(1 << (L - 1));
    E_f = v0f * (float)kFineDim;
    for (int l = 0; l < kMaxLevels; ++l) {
      v[l] = (R)v0f * (R)(1 << l);
      n[l] = kFineDim >> l;
    }
  }

  static size_t vox(int n, int x, int y, int z) { return (size_t)x + (size_t)n * ((size_t)y + (size_t)n * z); }

  // ---- allocation (Sec. 3.2): insert the blocks of a segment; new blocks start at the finest level (Sec. 3.2.1)
  void allocate(const std::vector<Key>& cells, std::set<Key>& touched, orc_frame_stats* st,
                std::vector<Key>* fresh = nullptr) {
    for (const Key& k : cells) {
      touched.insert(k);
      if (blocks.find(k) == blocks.end()) {
        st->new_blocks++;
        auto ar = archive.find(k);
        if (ar != archive.end()) {  // streamed back in: level and payload as they were archived
          blocks[k] = std::move(ar->second);
          archive.erase(ar);
          st->restored++;
          continue;
        }
        Block<R, Sto>& b = blocks[k];
        b.level = 0;
        b.resize(n[0], P.has_color != 0);
        if (fresh) fresh->push_back(k);
      }
    }
  }

  // ---- capacity-driven streaming (Sec. 3.3). Reading: before a frame, when some level holds more blocks than
  // `fraction` of its pool (float comparison of the counts), every block outside the frame's view moves to the archive
  // (level and payload kept): for a camera, a block whose circumscribed sphere misses the pinhole's view cone between
  // min and max depth; for a LiDAR scan, a block whose centre lies farther than `radius` from the scan origin. A block
  // the frame allocates again comes back from the archive as it was.
  bool stream_on = false;
  float stream_fraction = 0.0f, stream_radius = 0.0f;
  int64_t stream_max[3] = {0, 0, 0};
  std::map<Key, Block<R, Sto>> archive;

  bool stream_due() const {
    if (!stream_on) return false;
    int64_t cnt[3] = {0, 0, 0};
    for (auto& kv : blocks) cnt[kv.second.level]++;
    for (int l = 0; l < L; ++l)
      if ((float)cnt[l] > stream_fraction * (float)stream_max[l]) return true;
    return false;
  }
  void centre_of(const Key& k, float c[3]) const {
    c[0] = ((float)k.x + 0.5f) * E_f;
    c[1] = ((float)k.y + 0.5f) * E_f;
    c[2] = ((float)k.z + 0.5f) * E_f;
  }
  template <class Outside>
  void evict(Outside&& outside, orc_frame_stats* st) {
    for (auto it = blocks.begin(); it != blocks.end();) {
      float c[3];
      centre_of(it->first, c);
      if (outside(c)) {
        archive[it->first] = std::move(it->second);
        it = blocks.erase(it);
        st->evicted++;
      } else {
        ++it;
      }
    }
  }
  void stream_out_camera(const orc_pinhole* K, const float Rf[9], const float tf[3], orc_frame_stats* st) {
    if (!stream_due()) return;
    const float rad = 0.8660254f * E_f;
    const float tx = std::max(K->cx, (float)K->width - K->cx) / K->fx;
    const float ty = std::max(K->cy, (float)K->height - K->cy) / K->fy;
    const float kx = std::sqrt(1.0f + tx * tx), ky = std::sqrt(1.0f + ty * ty);
    evict([&](const float c[3]) {
      const float d0 = c[0] - tf[0], d1 = c[1] - tf[1], d2 = c[2] - tf[2];
      const float xc = Rf[0] * d0 + Rf[3] * d1 + Rf[6] * d2;
      const float yc = Rf[1] * d0 + Rf[4] * d1 + Rf[7] * d2;
      const float zc = Rf[2] * d0 + Rf[5] * d1 + Rf[8] * d2;
      const bool inside = zc + rad >= K->min_depth && zc - rad <= K->max_depth &&
                          std::fabs(xc) <= zc * tx + rad * kx && std::fabs(yc) <= zc * ty + rad * ky;
      return !inside;
    }, st);
  }
  void stream_out_lidar(const double* T, orc_frame_stats* st) {
    if (!stream_due()) return;
    const float o[3] = {(float)T[3], (float)T[7], (float)T[11]};
    const float r2 = stream_radius * stream_radius;
    evict([&](const float c[3]) {
      const float d0 = c[0] - o[0], d1 = c[1] - o[1], d2 = c[2] - o[2];
      return d0 * d0 + d1 * d1 + d2 * d2 > r2;
    }, st);
  }
  int64_t archived() const override { return (int64_t)archive.size(); }

  // ---- Eq. 3 with w_k = 1 in Welford's incremental form, and the Welford S2 update (Sec. 3.2.1).
  // The running mean D + (d - D)/(W + 1) equals (W D + d)/(W + 1) of Eq. 3 in exact arithmetic; this form keeps a
  // voxel that sees the same d again at exactly D, so its S2 stays exactly 0. Reading of the arithmetic: the division
  // by W + 1 is a multiplication by the correctly rounded reciprocal 1/(W + 1), shared by the distance and the colour
  // channels (the same quantity in exact arithmetic; one reciprocal per observation instead of four quotients).
  void update(Block<R, Sto>& b, size_t i, R d, const R* col) {
    R W = b.W[i];
    R D = (R)Store<Sto>::get(b.D[i]);
    R Wn = W + (R)1;
    R inv = (R)1 / Wn;
    R e = d - D;
    R Dn = D + e * inv;
    b.S2[i] = b.S2[i] + e * (d - Dn);
    b.D[i] = Store<Sto>::put(Dn);
    b.W[i] = Wn;
    if (col && P.has_color) {
      for (int c = 0; c < 3; ++c) {
        R C = (R)Store<Sto>::get(b.C[c][i]);
        R ec = col[c] - C;
        b.C[c][i] = Store<Sto>::put(C + ec * inv);
      }
    }
  }

  // ---- block statistics (Sec. 3.2.1: "aggregated at the block level to obtain the mean variance of each block").
  // Reading: the mean runs over observed voxels (W > 0); an unobserved voxel has no variance. Always double, voxel
  // index order.
  struct BStat {
    int64_t n_obs, sum_w;
    double vbar;
  };
  BStat stats(const Block<R, Sto>& b) const {
    BStat s{0, 0, 0.0};
    double acc = 0.0;
    size_t nv = b.W.size();
    for (size_t i = 0; i < nv; ++i) {
      if (b.W[i] > (R)0) {
        s.n_obs++;
        s.sum_w += (int64_t)b.W[i];
        acc += (double)b.S2[i] / (double)b.W[i];
      }
    }
    s.vbar = s.n_obs ? acc / (double)s.n_obs : 0.0;
    return s;
  }

  // ---- merge l -> l+1 (Sec. 3.2.1, Fig. 4a: a low-variance block is re-allocated at a coarser resolution).
  // Reading: each coarse voxel pools its 2x2x2 observed children: D and colour are W-weighted means, sigma^2 is the
  // W-weighted mean of child variances, W is the largest child weight, S2 = sigma^2 W.
  void merge(Block<R, Sto>& b) {
    int nf = n[b.level], nc = nf / 2;
    Block<R, Sto> c;
    c.level = b.level + 1;
    c.resize(nc, P.has_color != 0);
    for (int z = 0; z < nc; ++z)
      for (int y = 0; y < nc; ++y)
        for (int x = 0; x < nc; ++x) {
          R sw = 0, swd = 0, ss2 = 0, wmax = 0, swc[3] = {0, 0, 0};
          for (int k = 0; k < 8; ++k) {
            size_t ch = vox(nf, 2 * x + (k & 1), 2 * y + ((k >> 1) & 1), 2 * z + (k >> 2));
            R Wi = b.W[ch];
            if (!(Wi > (R)0)) continue;
            sw = sw + Wi;
            swd = swd + Wi * (R)Store<Sto>::get(b.D[ch]);
            ss2 = ss2 + b.S2[ch];
            if (Wi > wmax) wmax = Wi;
            if (P.has_color)
              for (int q = 0; q < 3; ++q) swc[q] = swc[q] + Wi * (R)Store<Sto>::get(b.C[q][ch]);
          }
          size_t o = vox(nc, x, y, z);
          if (sw > (R)0) {
            R var = ss2 / sw;
            c.D[o] = Store<Sto>::put(swd / sw);
            c.W[o] = wmax;
            c.S2[o] = var * wmax;
            if (P.has_color)
              for (int q = 0; q < 3; ++q) c.C[q][o] = Store<Sto>::put(swc[q] / sw);
          }
        }
    b = std::move(c);
  }

  // ---- split l -> l-1 (extension: the inverse of the merge, for blocks whose variance has grown again).
  // Reading: each fine voxel takes the trilinear interpolation of the coarse D and colour at its centre over observed
  // coarse voxels of this block (clamped to the block, weights renormalised); W and S2 are copied from the coarse
  // voxel that contains it.
  void split(Block<R, Sto>& b) {
    int nc = n[b.level], nf = nc * 2;
    Block<R, Sto> f;
    f.level = b.level - 1;
    f.resize(nf, P.has_color != 0);
    for (int z = 0; z < nf; ++z)
      for (int y = 0; y < nf; ++y)
        for (int x = 0; x < nf; ++x) {
          int fi[3] = {x, y, z}, i0[3];
          R fr[3];
          for (int a = 0; a < 3; ++a) {
            R p = (R)fi[a] * (R)0.5 - (R)0.25;  // fine centre in coarse voxel-index coordinates
            if (p < (R)0) p = (R)0;
            if (p > (R)(nc - 1)) p = (R)(nc - 1);
            int i = (int)std::floor(p);
            if (i > nc - 2) i = nc - 2;
            i0[a] = i;
            fr[a] = p - (R)i;
          }
          R sw = 0, sd = 0, sc[3] = {0, 0, 0};
          for (int k = 0; k < 8; ++k) {
            int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
            size_t cv = vox(nc, i0[0] + ax, i0[1] + ay, i0[2] + az);
            if (!(b.W[cv] > (R)0)) continue;
            R wx = ax ? fr[0] : (R)1 - fr[0];
            R wy = ay ? fr[1] : (R)1 - fr[1];
            R wz = az ? fr[2] : (R)1 - fr[2];
            R w = (wx * wy) * wz;
            sw = sw + w;
            sd = sd + w * (R)Store<Sto>::get(b.D[cv]);
            if (P.has_color)
              for (int q = 0; q < 3; ++q) sc[q] = sc[q] + w * (R)Store<Sto>::get(b.C[q][cv]);
          }
          size_t own = vox(nc, x >> 1, y >> 1, z >> 1);
          size_t o = vox(nf, x, y, z);
          if (sw > (R)0) {
            f.D[o] = Store<Sto>::put(sd / sw);
            if (P.has_color)
              for (int q = 0; q < 3; ++q) f.C[q][o] = Store<Sto>::put(sc[q] / sw);
          } else {
            f.D[o] = b.D[own];
            if (P.has_color)
              for (int q = 0; q < 3; ++q) f.C[q][o] = b.C[q][own];
          }
          f.W[o] = b.W[own];
          f.S2[o] = b.S2[own];
        }
    b = std::move(f);
  }

  // ---- re-level every touched block once (Sec. 3.2.1). Reading: a block may change level only after its observed
  // voxels carry a mean weight of at least k_min (one frame gives S2 = 0 everywhere), and at most once per frame.
  void relevel(const std::set<Key>& touched, orc_frame_stats* st) {
    for (const Key& k : touched) {
      Block<R, Sto>& b = blocks[k];
      BStat s = stats(b);
      if (s.n_obs == 0) continue;
      if (s.sum_w < (int64_t)P.min_obs * s.n_obs) continue;
      if (b.level < L - 1 && s.vbar < P.var_threshold[b.level]) {
        merge(b);
        st->merged++;
      } else if (P.split_hysteresis > 0.0 && b.level > 0 &&
                 s.vbar > P.split_hysteresis * P.var_threshold[b.level - 1]) {
        split(b);
        st->split++;
      }
    }
  }

  // ---- pose as float (f32s) or double (f64) rotation + translation
  void pose(const double* T, R Rm[9], R t[3]) const {
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) Rm[3 * r + c] = (R)T[4 * r + c];
      t[r] = (R)T[4 * r + 3];
    }
  }

  // ---- camera integration (Sec. 3.1.2, Eq. 2)
  int integrate_depth(const orc_pinhole* K, const double* T, const float* depth, const uint8_t* rgb,
                      orc_frame_stats* st) override {
    std::memset(st, 0, sizeof(*st));
    // (1) rays and allocation. The key endpoints always follow this float sequence.
    float Rf[9], tf[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) Rf[3 * r + c] = (float)T[4 * r + c];
      tf[r] = (float)T[4 * r + 3];
    }
    const float tauf = P.truncation;
    const float Sfix = 65536.0f / E_f;
    stream_out_camera(K, Rf, tf, st);
    std::set<Key> touched;
    std::vector<Key> fresh;  // blocks created by this frame
    for (int v_ = 0; v_ < K->height; ++v_) {
      for (int u = 0; u < K->width; ++u) {
        float z = depth[(size_t)v_ * K->width + u];
        if (!(z >= K->min_depth && z <= K->max_depth)) continue;
        float qx = ((float)u - K->cx) / K->fx;
        float qy = ((float)v_ - K->cy) / K->fy;
        float nq = std::sqrt(qx * qx + qy * qy + 1.0f);
        float rho = z * nq;
        float rc[3] = {qx / nq, qy / nq, 1.0f / nq};
        float r[3];
        for (int a = 0; a < 3; ++a) r[a] = Rf[3 * a + 0] * rc[0] + Rf[3 * a + 1] * rc[1] + Rf[3 * a + 2] * rc[2];
        float t0 = rho - tauf;
        if (t0 < 0.0f) t0 = 0.0f;
        float t1 = rho + tauf;
        int64_t A[3], B[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
          ok = ok && to_fixed_f(tf[a] + t0 * r[a], Sfix, &A[a]);
          ok = ok && to_fixed_f(tf[a] + t1 * r[a], Sfix, &B[a]);
        }
        if (!ok) continue;
        Key ka{floor_div(A[0], kBlockUnit), floor_div(A[1], kBlockUnit), floor_div(A[2], kBlockUnit)};
        Key kb{floor_div(B[0], kBlockUnit), floor_div(B[1], kBlockUnit), floor_div(B[2], kBlockUnit)};
        if (!key_in_range(ka) || !key_in_range(kb)) continue;
        st->valid_rays++;
        allocate(cells_bruteforce(A, B, kBlockUnit), touched, st, &fresh);
      }
    }
    st->touched = (int64_t)touched.size();
    // (1b) learned level predictor (not in the paper): a new block starts at the level predicted from its features
    // in this frame's range image instead of the finest level; capture records the features as training data.
    if (!pred_w.empty() || capture) {
      std::vector<float> rho_img((size_t)K->width * K->height, -1.0f);
      for (int v_ = 0; v_ < K->height; ++v_)
        for (int u = 0; u < K->width; ++u) {
          float z = depth[(size_t)v_ * K->width + u];
          if (!(z >= K->min_depth && z <= K->max_depth)) continue;
          float qx = ((float)u - K->cx) / K->fx;
          float qy = ((float)v_ - K->cy) / K->fy;
          rho_img[(size_t)v_ * K->width + u] = z * std::sqrt(qx * qx + qy * qy + 1.0f);
        }
      for (const Key& k : fresh) {
        float f[16];
        int lvl = -1;
        if (!orc_block_features(K, Rf, tf, rho_img.data(), E_f, P.truncation, k.x, k.y, k.z,
                                pred_w.empty() ? nullptr : pred_w.data(), L, f, &lvl))
          continue;
        if (lvl > 0) {
          Block<R, Sto>& b = blocks[k];
          b.level = lvl;
          b.resize(n[lvl], P.has_color != 0);
        }
        if (capture) {
          cap_keys.push_back(k);
          cap_feat.insert(cap_feat.end(), f, f + 16);
        }
      }
    }
    // (2) projective fusion of every voxel of every touched block.
    R Rm[9], t[3];
    pose(T, Rm, t);
    const R fx = (R)K->fx, fy = (R)K->fy, cx = (R)K->cx, cy = (R)K->cy;
    const R E = (R)E_f;
    for (const Key& k : touched) {
      Block<R, Sto>& b = blocks[k];
      int l = b.level, nl = n[l];
      R vl = v[l];
      R ob[3] = {(R)k.x * E - t[0], (R)k.y * E - t[1], (R)k.z * E - t[2]};  // block corner relative to the camera
      for (int zi = 0; zi < nl; ++zi)
        for (int yi = 0; yi < nl; ++yi)
          for (int xi = 0; xi < nl; ++xi) {
            R w[3] = {ob[0] + ((R)xi + (R)0.5) * vl, ob[1] + ((R)yi + (R)0.5) * vl, ob[2] + ((R)zi + (R)0.5) * vl};
            R xc = Rm[0] * w[0] + Rm[3] * w[1] + Rm[6] * w[2];
            R yc = Rm[1] * w[0] + Rm[4] * w[1] + Rm[7] * w[2];
            R zc = Rm[2] * w[0] + Rm[5] * w[1] + Rm[8] * w[2];
            if (!(zc > (R)0)) continue;
            // Eq. 2's projection pi(x), nearest pixel; the two quotients by z use its correctly rounded reciprocal
            R iz = (R)1 / zc;
            R uf = fx * xc * iz + cx + (R)0.5;
            R vf = fy * yc * iz + cy + (R)0.5;
            if (!(uf >= (R)0 && uf < (R)K->width && vf >= (R)0 && vf < (R)K->height)) continue;
            int u = (int)std::floor(uf), vv = (int)std::floor(vf);
            size_t pix = (size_t)vv * K->width + u;
            float zm = depth[pix];
            if (!(zm >= K->min_depth && zm <= K->max_depth)) continue;
            R qx = ((R)u - cx) / fx, qy = ((R)vv - cy) / fy;
            R rho = (R)zm * std::sqrt(qx * qx + qy * qy + (R)1);
            R dist = std::sqrt(xc * xc + yc * yc + zc * zc);
            // Eq. 2: d = rho - |x|. Reading: rho is the measured range along the pixel ray (z-depth times the ray
            // length at unit z), so both terms are ranges. A voxel more than tau behind the surface is occluded and
            // not updated; otherwise d is clipped to tau.
            R eta = rho - dist;
            if (eta < -tau) continue;
            R d = eta < tau ? eta : tau;
            R col[3];
            if (rgb) for (int q = 0; q < 3; ++q) col[q] = (R)rgb[3 * pix + q];
            update(b, vox(nl, xi, yi, zi), d, rgb ? col : nullptr);
            st->observations++;
          }
    }
    // (3) block variance and re-levelling (a camera frame observes a voxel at most once)
    st->updated_voxels = st->observations;
    relevel(touched, st);
    return 0;
  }

  // ---- LiDAR integration (Sec. 3.1.1, Eq. 1)
  int integrate_points(const double* T, const float* xyz, int64_t npts, orc_frame_stats* st) override {
    std::memset(st, 0, sizeof(*st));
    stream_out_lidar(T, st);
    const double tau_d = (double)P.truncation;
    const double Sfix = 65536.0 / (double)E_f;
    const double rmin2 = (double)P.min_range * (double)P.min_range, rmax2 = (double)P.max_range * (double)P.max_range;
    struct RayRec {
      int64_t A[3], B[3];
      double rho, rhat[3];
    };
    std::vector<RayRec> rays;
    std::vector<int64_t> ray_index;
    std::set<Key> touched;
    std::vector<Key> fresh;  // blocks created by this scan
    std::vector<std::array<int64_t, 3>> ends;  // end points of the valid rays (fixed point), when one converts
    // (1) rays (double) and allocation
    for (int64_t j = 0; j < npts; ++j) {
      double xs[3] = {(double)xyz[3 * j], (double)xyz[3 * j + 1], (double)xyz[3 * j + 2]};
      double n2 = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
      if (!(n2 >= rmin2 && n2 <= rmax2)) continue;
      double p[3], dv[3];
      for (int a = 0; a < 3; ++a) {
        p[a] = T[4 * a + 0] * xs[0] + T[4 * a + 1] * xs[1] + T[4 * a + 2] * xs[2] + T[4 * a + 3];
        dv[a] = p[a] - T[4 * a + 3];
      }
      // length and direction of the ray in float (reading: FP64 is confined to the pose composition above and the
      // fixed-point band ends below)
      RayRec rr;
      const float d0 = (float)dv[0], d1 = (float)dv[1], d2 = (float)dv[2];
      const float rf = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      rr.rho = (double)rf;
      rr.rhat[0] = (double)(d0 / rf);
      rr.rhat[1] = (double)(d1 / rf);
      rr.rhat[2] = (double)(d2 / rf);
      double t0 = rr.rho - tau_d;
      if (t0 < 0.0) t0 = 0.0;
      double t1 = rr.rho + tau_d;
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        ok = ok && to_fixed_d(T[4 * a + 3] + t0 * rr.rhat[a], Sfix, &rr.A[a]);
        ok = ok && to_fixed_d(T[4 * a + 3] + t1 * rr.rhat[a], Sfix, &rr.B[a]);
      }
      if (!ok) continue;
      Key ka{floor_div(rr.A[0], kBlockUnit), floor_div(rr.A[1], kBlockUnit), floor_div(rr.A[2], kBlockUnit)};
      Key kb{floor_div(rr.B[0], kBlockUnit), floor_div(rr.B[1], kBlockUnit), floor_div(rr.B[2], kBlockUnit)};
      if (!key_in_range(ka) || !key_in_range(kb)) continue;
      st->valid_rays++;
      allocate(cells_bruteforce(rr.A, rr.B, kBlockUnit), touched, st, &fresh);
      rays.push_back(rr);
      ray_index.push_back(j);
      std::array<int64_t, 3> e;
      if (to_fixed_d(p[0], Sfix, &e[0]) && to_fixed_d(p[1], Sfix, &e[1]) && to_fixed_d(p[2], Sfix, &e[2]))
        ends.push_back(e);
    }
    st->touched = (int64_t)touched.size();
    // (1b) learned level predictor (not in the paper): a new block starts at the level predicted from the moments of
    // the scan's end points inside it (position in the block quantised to 1/1024 of its edge) instead of the finest
    // level; capture records the features as training data.
    if (!pred_w.empty() || capture) {
      std::map<Key, std::array<uint64_t, 10>> mom;
      for (const Key& k : fresh) mom[k].fill(0);
      for (const auto& e : ends) {
        Key k{floor_div(e[0], kBlockUnit), floor_div(e[1], kBlockUnit), floor_div(e[2], kBlockUnit)};
        auto it = mom.find(k);
        if (it == mom.end()) continue;
        const int64_t kc[3] = {k.x, k.y, k.z};
        uint64_t q[3];  // 0 <= e - k E < E, in units of E / 1024
        for (int a = 0; a < 3; ++a) q[a] = (uint64_t)((e[a] - kc[a] * kBlockUnit) / (kBlockUnit / 1024));
        std::array<uint64_t, 10>& M = it->second;
        M[0] += 1;
        for (int a = 0; a < 3; ++a) M[1 + a] += q[a];
        for (int a = 0; a < 3; ++a) M[4 + a] += q[a] * q[a];
        M[7] += q[0] * q[1];
        M[8] += q[0] * q[2];
        M[9] += q[1] * q[2];
      }
      for (const Key& k : fresh) {
        float f[16];
        int lvl = -1;
        orc_lidar_block_features(mom[k].data(), T, E_f, P.truncation, k.x, k.y, k.z,
                                 pred_w.empty() ? nullptr : pred_w.data(), L, f, &lvl);
        if (lvl > 0) {
          Block<R, Sto>& b = blocks[k];
          b.level = lvl;
          b.resize(n[lvl], P.has_color != 0);
        }
        if (capture) {
          cap_keys.push_back(k);
          cap_feat.insert(cap_feat.end(), f, f + 16);
        }
      }
    }
    // (2) ray-based fusion: each ray walks the voxels of its truncation band in ascending point index; a voxel at
    // level l is observed once per ray that crosses it (any of its finest-level cells).
    R Rm[9], t[3];
    pose(T, Rm, t);
    (void)Rm;
    const R E = (R)E_f;
    std::unordered_set<uint64_t> updated;  // (block, voxel) pairs updated by this scan
    for (size_t q = 0; q < rays.size(); ++q) {
      const RayRec& rr = rays[q];
      std::vector<Key> fine = cells_dda(rr.A, rr.B, kVoxelUnit);
      R rho = (R)rr.rho;
      R rh[3] = {(R)rr.rhat[0], (R)rr.rhat[1], (R)rr.rhat[2]};
      bool have_prev = false;
      Key prev_b{0, 0, 0};
      int64_t prev_g[3] = {0, 0, 0};
      for (const Key& f : fine) {
        Key bk{floor_div(f.x, kFineDim), floor_div(f.y, kFineDim), floor_div(f.z, kFineDim)};
        auto it = blocks.find(bk);
        if (it == blocks.end()) continue;
        Block<R, Sto>& b = it->second;
        int l = b.level;
        int64_t g[3] = {floor_div(f.x, (int64_t)1 << l), floor_div(f.y, (int64_t)1 << l),
                        floor_div(f.z, (int64_t)1 << l)};
        if (have_prev && prev_b == bk && prev_g[0] == g[0] && prev_g[1] == g[1] && prev_g[2] == g[2]) continue;
        have_prev = true;
        prev_b = bk;
        std::memcpy(prev_g, g, sizeof(g));
        int nl = n[l];
        int li[3] = {(int)(g[0] - bk.x * nl), (int)(g[1] - bk.y * nl), (int)(g[2] - bk.z * nl)};
        // Eq. 1: d = clip((p - x) . n, -tau, tau). With p = o + rho n and |n| = 1 this is rho - (x - o) . n.
        R xr[3];
        R ob[3] = {(R)bk.x * E - t[0], (R)bk.y * E - t[1], (R)bk.z * E - t[2]};
        for (int a = 0; a < 3; ++a) xr[a] = ob[a] + ((R)li[a] + (R)0.5) * v[l];
        R d = rho - (xr[0] * rh[0] + xr[1] * rh[1] + xr[2] * rh[2]);
        if (d < -tau) d = -tau;
        if (d > tau) d = tau;
        update(b, vox(nl, li[0], li[1], li[2]), d, nullptr);
        updated.insert((uint64_t)(uintptr_t)&b * 1024u + (uint64_t)vox(nl, li[0], li[1], li[2]));
        st->observations++;
      }
    }
    st->updated_voxels = (int64_t)updated.size();
    relevel(touched, st);
    return 0;
  }

  // ---- raycast (the rendering branch of Fig. 2; the paper renders through Gaussian splats and gives no raycaster).
  // Definition: along the ray of pixel (u, v), between min_depth and max_depth (as z-depth), the first place where the
  // trilinear TSDF passes from positive to non-positive. The field F(x) exists where the block holding x is allocated
  // and the 8 voxel centres of that block's level nearest to x are all observed (W > 0); a corner is read from the
  // block holding the corner centre, from that block's voxel containing it, whatever the block's level. Everything
  // here is double arithmetic on the stored values, in both modes.
  // Search: samples on the grid t_j = t_min + j h, with h = min(v_0, tau / 2) (the sampling step of the finest
  // level). A level-l block is sampled at its own voxel pitch, min(v_l, tau / 2): every 2^l-th grid sample from its
  // first one, and the first grid sample past its exit face follows in any case. Two consecutive samples that both
  // have a field, with F > 0 at the first and F <= 0 at the second, bracket the crossing; the first such bracket is
  // narrowed by bisection below 1e-9 m and the crossing is the linear root of the last bracket (a midpoint without a
  // field ends the bisection at that midpoint). A grid sample in an unallocated block has no field, and neither has
  // any other sample of that block, so the search continues at the first grid sample past the block's exit face.
  // Output z-depth, 0 where there is no crossing; optionally the normal and colour at the crossing (shade_at()).
  static constexpr double kRayBisectTol = 1e-9;  // bracket width [m] at which the bisection stops

  // Block lookups of one ray, remembered (the same block answers most corner lookups in a row).
  struct Lookup {
    const Map* map;
    Key k[2];
    const Block<R, Sto>* b[2] = {nullptr, nullptr};
    bool have[2] = {false, false};
    const Block<R, Sto>* get(const Key& key) {
      for (int i = 0; i < 2; ++i)
        if (have[i] && k[i] == key) return b[i];
      k[1] = k[0];
      b[1] = b[0];
      have[1] = have[0];
      auto it = map->blocks.find(key);
      k[0] = key;
      b[0] = it == map->blocks.end() ? nullptr : &it->second;
      have[0] = true;
      return b[0];
    }
  };

  const Block<R, Sto>* find(const Key& k) const {
    auto it = blocks.find(k);
    return it == blocks.end() ? nullptr : &it->second;
  }

  double vd(int l) const { return (double)(E_f / (float)kFineDim) * (double)(1 << l); }  // voxel edge of level l

  // the 8 corners of x on the level-l grid: block, voxel index and trilinear weight of each (corner k has offset
  // (k & 1, (k >> 1) & 1, k >> 2)); false when a corner's block is unallocated or the corner is unobserved
  bool corners(Lookup& lk, const double x[3], int l, const Block<R, Sto>* cb[8], size_t ci[8], double cw[8],
               double fr[3]) const {
    const double vl = vd(l);
    int64_t j0[3];
    for (int a = 0; a < 3; ++a) {
      const double g = x[a] / vl - 0.5;
      const double fl = std::floor(g);
      j0[a] = (int64_t)fl;
      fr[a] = g - fl;
    }
    const int nl = n[l];
    for (int k = 0; k < 8; ++k) {
      const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
      const int64_t j[3] = {j0[0] + ax, j0[1] + ay, j0[2] + az};
      const Key bk{floor_div(j[0], nl), floor_div(j[1], nl), floor_div(j[2], nl)};
      const Block<R, Sto>* b = lk.get(bk);
      if (!b) return false;
      size_t idx;
      if (b->level == l) {
        idx = vox(nl, (int)(j[0] - bk.x * nl), (int)(j[1] - bk.y * nl), (int)(j[2] - bk.z * nl));
      } else {
        // the finest-level cell holding the corner centre, then the voxel of block bk's level containing it
        const int lb = b->level, nb = n[lb];
        int64_t cf[3];
        for (int a = 0; a < 3; ++a) cf[a] = l == 0 ? j[a] : j[a] * ((int64_t)1 << l) + ((int64_t)1 << (l - 1));
        idx = vox(nb, (int)(floor_div(cf[0], (int64_t)1 << lb) - bk.x * nb),
                  (int)(floor_div(cf[1], (int64_t)1 << lb) - bk.y * nb),
                  (int)(floor_div(cf[2], (int64_t)1 << lb) - bk.z * nb));
      }
      if (!((double)b->W[idx] > 0.0)) return false;
      cb[k] = b;
      ci[k] = idx;
      cw[k] = (ax ? fr[0] : 1.0 - fr[0]) * (ay ? fr[1] : 1.0 - fr[1]) * (az ? fr[2] : 1.0 - fr[2]);
    }
    return true;
  }

  // F at x: false when x's block is unallocated or the field does not exist there
  bool field_at(Lookup& lk, const double x[3], double* F) const {
    const double E = (double)E_f;
    const Block<R, Sto>* b =
        lk.get(Key{(int64_t)std::floor(x[0] / E), (int64_t)std::floor(x[1] / E), (int64_t)std::floor(x[2] / E)});
    if (!b) return false;
    const Block<R, Sto>* cb[8];
    size_t ci[8];
    double cw[8], fr[3];
    if (!corners(lk, x, b->level, cb, ci, cw, fr)) return false;
    double acc = 0.0;
    for (int k = 0; k < 8; ++k) acc += cw[k] * (double)Store<Sto>::get(cb[k]->D[ci[k]]);
    *F = acc;
    return true;
  }

  // Surface attributes at x, over the 8 corners of the level of x's block: g = the gradient of the trilinear
  // interpolant (times v_l: the derivative of a corner's weight along axis a is the product of its other two weights,
  // + for the upper corner, - for the lower), c = the trilinear mean of the stored colour. False when x's block is
  // unallocated or a corner is missing or unobserved.
  bool shade_at(Lookup& lk, const double x[3], double g[3], double c[3]) const {
    const double E = (double)E_f;
    for (int a = 0; a < 3; ++a) g[a] = c[a] = 0.0;
    const Block<R, Sto>* b =
        lk.get(Key{(int64_t)std::floor(x[0] / E), (int64_t)std::floor(x[1] / E), (int64_t)std::floor(x[2] / E)});
    if (!b) return false;
    const Block<R, Sto>* cb[8];
    size_t ci[8];
    double cw[8], fr[3];
    if (!corners(lk, x, b->level, cb, ci, cw, fr)) return false;
    for (int k = 0; k < 8; ++k) {
      const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
      const double wx = ax ? fr[0] : 1.0 - fr[0], wy = ay ? fr[1] : 1.0 - fr[1], wz = az ? fr[2] : 1.0 - fr[2];
      const double d = (double)Store<Sto>::get(cb[k]->D[ci[k]]);
      g[0] += (ax ? 1.0 : -1.0) * wy * wz * d;
      g[1] += (ay ? 1.0 : -1.0) * wx * wz * d;
      g[2] += (az ? 1.0 : -1.0) * wx * wy * d;
      if (P.has_color)
        for (int q = 0; q < 3; ++q) c[q] += cw[k] * (double)Store<Sto>::get(cb[k]->C[q][ci[k]]);
    }
    return true;
  }

  // unit normal and u8 colour at x (zeros when shade_at fails); returns whether it succeeded
  bool surface(Lookup& lk, const double x[3], float* normal, uint8_t* rgb) const {
    double g[3], c[3];
    const bool ok = shade_at(lk, x, g, c);
    if (normal) {
      const double nn = ok ? std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : 0.0;
      for (int a = 0; a < 3; ++a) normal[a] = nn > 0.0 ? (float)(g[a] / nn) : 0.0f;
    }
    if (rgb)
      for (int q = 0; q < 3; ++q) {
        const double cv = ok ? std::floor(c[q] + 0.5) : 0.0;
        rgb[q] = (uint8_t)(cv <= 0.0 ? 0 : cv >= 255.0 ? 255 : (int)cv);
      }
    return ok;
  }

  // One pixel: the crossing's ray parameter t (0 = none); rc = unit ray in the camera frame, r = in the world.
  double cast(const orc_pinhole* K, const double Rm[9], const double o[3], int u, int vv, double rc[3],
              double r[3]) const {
    const double qx = ((double)u - (double)K->cx) / (double)K->fx, qy = ((double)vv - (double)K->cy) / (double)K->fy;
    const double nq = std::sqrt(qx * qx + qy * qy + 1.0);
    rc[0] = qx / nq;
    rc[1] = qy / nq;
    rc[2] = 1.0 / nq;
    for (int a = 0; a < 3; ++a) r[a] = Rm[3 * a + 0] * rc[0] + Rm[3 * a + 1] * rc[1] + Rm[3 * a + 2] * rc[2];
    const double E = (double)E_f, h = std::min(vd(0), 0.5 * (double)tau);
    const double t_min = (double)K->min_depth * nq, t_max = (double)K->max_depth * nq;
    Lookup lk{this};
    bool have_prev = false;
    double t_prev = 0.0, F_prev = 0.0;
    for (int64_t j = 0;;) {
      const double t = t_min + (double)j * h;
      if (t > t_max) return 0.0;
      const double x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
      const Key bk{(int64_t)std::floor(x[0] / E), (int64_t)std::floor(x[1] / E), (int64_t)std::floor(x[2] / E)};
      if (!lk.get(bk)) {
        // no sample of this block has a field: continue at the first grid sample past its exit face
        double t_exit = t_max + 1.0;
        for (int a = 0; a < 3; ++a) {
          if (r[a] == 0.0) continue;
          const double face = (double)(r[a] > 0.0 ? (&bk.x)[a] + 1 : (&bk.x)[a]) * E;
          t_exit = std::min(t_exit, (face - o[a]) / r[a]);
        }
        const int64_t jn = (int64_t)std::ceil((t_exit - t_min) / h);
        j = jn > j ? jn : j + 1;
        have_prev = false;
        continue;
      }
      const Block<R, Sto>* blk = lk.get(bk);
      double F = 0.0;
      const bool valid = field_at(lk, x, &F);
      if (valid && have_prev && F_prev > 0.0 && !(F > 0.0)) {
        double a = t_prev, b = t, Fa = F_prev, Fb = F;
        while (b - a > kRayBisectTol) {
          const double m = 0.5 * (a + b);
          const double xm[3] = {o[0] + m * r[0], o[1] + m * r[1], o[2] + m * r[2]};
          double Fm = 0.0;
          if (!field_at(lk, xm, &Fm)) return m;  // the bracket holds a point without a field: stop there
          if (Fm > 0.0) {
            a = m;
            Fa = Fm;
          } else {
            b = m;
            Fb = Fm;
          }
        }
        return a + (b - a) * (Fa / (Fa - Fb));  // the linear root of the final bracket (exact on a linear field)
      }
      have_prev = valid;
      t_prev = t;
      F_prev = F;
      if (blk->level > 0) {
        // a level-l block is sampled every 2^l grid steps (its own voxel pitch), counted from its first sample; the
        // first sample past its exit face is taken in any case
        double t_exit = t_max + 1.0;
        for (int a = 0; a < 3; ++a) {
          if (r[a] == 0.0) continue;
          const double face = (double)(r[a] > 0.0 ? (&bk.x)[a] + 1 : (&bk.x)[a]) * E;
          t_exit = std::min(t_exit, (face - o[a]) / r[a]);
        }
        const int64_t jn = (int64_t)std::ceil((t_exit - t_min) / h);
        const int64_t step = std::min((int64_t)1 << blk->level, jn > j ? jn - j : (int64_t)1);
        j += step;
        continue;
      }
      ++j;
    }
  }

  void pose_d(const double* T, double Rm[9], double o[3]) const {
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) Rm[3 * a + b] = T[4 * a + b];
      o[a] = T[4 * a + 3];
    }
  }

  // pixels pix[0 .. n) (index v * width + u) into depth[i], normal[3 i], rgb[3 i]
  int raycast_pixels(const orc_pinhole* K, const double* T, int64_t n_pix, const int64_t* pix, float* out,
                     float* normal, uint8_t* rgb) const override {
    double Rm[9], o[3];
    pose_d(T, Rm, o);
    for (int64_t i = 0; i < n_pix; ++i) {
      const int u = (int)(pix[i] % K->width), vv = (int)(pix[i] / K->width);
      double rc[3], r[3];
      const double t = cast(K, Rm, o, u, vv, rc, r);
      out[i] = (float)(t * rc[2]);
      if (normal || rgb) {
        float nz[3] = {0.0f, 0.0f, 0.0f};
        uint8_t cz[3] = {0, 0, 0};
        if (t > 0.0) {
          Lookup lk{this};
          const double xh[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
          surface(lk, xh, normal ? nz : nullptr, rgb ? cz : nullptr);
        }
        if (normal) std::memcpy(normal + 3 * i, nz, sizeof nz);
        if (rgb) std::memcpy(rgb + 3 * i, cz, sizeof cz);
      }
    }
    return 0;
  }

  int raycast(const orc_pinhole* K, const double* T, float* out, float* normal, uint8_t* rgb) override {
    const int64_t np = (int64_t)K->width * K->height;
    std::vector<int64_t> pix((size_t)np);
    for (int64_t i = 0; i < np; ++i) pix[(size_t)i] = i;
    return raycast_pixels(K, T, np, pix.data(), out, normal, rgb);
  }

  // test hook: F at world points (valid[i] = 0 where it does not exist), and normal / colour there
  void probe_points(int64_t n_pts, const double* xyz, double* F, int8_t* valid, float* normal,
                    uint8_t* rgb) const override {
    Lookup lk{this};
    for (int64_t i = 0; i < n_pts; ++i) {
      double f = 0.0;
      const bool ok = field_at(lk, xyz + 3 * i, &f);
      if (F) F[i] = ok ? f : 0.0;
      if (valid) valid[i] = ok ? 1 : 0;
      if (normal || rgb) surface(lk, xyz + 3 * i, normal ? normal + 3 * i : nullptr, rgb ? rgb + 3 * i : nullptr);
    }
  }

  void set_streaming(float fraction, float radius, const int64_t* max_blocks) override {
    stream_on = fraction > 0.0f;
    stream_fraction = fraction;
    stream_radius = radius;
    for (int l = 0; l < 3; ++l) stream_max[l] = max_blocks[l];
  }

  // ---- test hook: write one block (created at `level` if missing) with the given payload
  int set_block(const int32_t* key, int level, const double* D, const double* W, const double* S2,
                const double* C) override {
    if (level < 0 || level >= L) return -1;
    Key k{key[0], key[1], key[2]};
    Block<R, Sto>& b = blocks[k];
    b.level = level;
    b.resize(n[level], P.has_color != 0);
    for (size_t i = 0; i < b.W.size(); ++i) {
      b.D[i] = Store<Sto>::put((R)D[i]);
      b.W[i] = (R)W[i];
      b.S2[i] = (R)S2[i];
      if (P.has_color && C)
        for (int q = 0; q < 3; ++q) b.C[q][i] = Store<Sto>::put((R)C[3 * i + q]);
    }
    return 0;
  }

  // ---- multi-resolution Marching Cubes (Sec. 3.4, Figs. 5 and 6). Reading: positions are
  // integers in units of half a finest voxel (a block edge is 2 n_0 units; a level-l voxel centre lies at an odd
  // multiple of 2^l). Every voxel of every block is the low corner of one cell, which runs along each axis to the next
  // voxel centre: inside the block one voxel further; from the block's last voxel, to the first centre of the
  // neighbouring block (half a voxel of each level), so a coarse cell next to a finer block is cut short and the two
  // blocks' cells tile space without overlap (the "truncated" coarse voxels); no cell where that neighbour is
  // missing. A cell corner's value is the trilinear field at the corner on the grid of the block that contains it,
  // each of the 8 nearest centres read from the voxel that contains it, whatever its block's level (coarse and fine
  // values blend across resolution boundaries); corners of zero weight are not read. A cell with an unallocated or
  // unobserved corner read emits nothing. The surface crossing on an edge is linear between its two corner values.
  bool mc_value(const int64_t P[3], R* out) const {
    const int64_t bu = 2 * kFineDim;
    const Block<R, Sto>* b = find(Key{floor_div(P[0], bu), floor_div(P[1], bu), floor_div(P[2], bu)});
    if (!b) return false;
    const int64_t s = (int64_t)1 << b->level, s2 = 2 * s;
    int64_t j0[3];
    R fr[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t g = P[a] - s;
      j0[a] = floor_div(g, s2);
      fr[a] = (R)(g - j0[a] * s2) / (R)s2;
    }
    R acc = 0;
    for (int k = 0; k < 8; ++k) {
      const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
      const R wx = ax ? fr[0] : (R)1 - fr[0];
      const R wy = ay ? fr[1] : (R)1 - fr[1];
      const R wz = az ? fr[2] : (R)1 - fr[2];
      const R w = (wx * wy) * wz;
      if (w == (R)0) continue;
      const int bit[3] = {ax, ay, az};
      int64_t C[3];
      for (int a = 0; a < 3; ++a) C[a] = (2 * (j0[a] + bit[a]) + 1) * s;
      const Key kc{floor_div(C[0], bu), floor_div(C[1], bu), floor_div(C[2], bu)};
      const Block<R, Sto>* bc = find(kc);
      if (!bc) return false;
      const int64_t vu = (int64_t)2 << bc->level;
      const int nb = n[bc->level];
      const size_t idx = vox(nb, (int)((C[0] - kc.x * bu) / vu), (int)((C[1] - kc.y * bu) / vu),
                             (int)((C[2] - kc.z * bu) / vu));
      if (!(bc->W[idx] > (R)0)) return false;
      acc = acc + w * (R)Store<Sto>::get(bc->D[idx]);
    }
    *out = acc;
    return true;
  }

  // triangle soup, 9 coordinates per triangle, blocks in key order and voxels in index order
  void extract_mesh(std::vector<float>& tris) const {
    static const McTable tab;
    const int64_t bu = 2 * kFineDim;
    const R unit = (R)(E_f / (float)bu);
    for (const Key& k : sorted_keys()) {
      const Block<R, Sto>& b = blocks.at(k);
      const int l = b.level, nl = n[l];
      const int64_t s = (int64_t)1 << l;
      const int64_t K[3] = {k.x, k.y, k.z};
      int64_t h_last[3];
      bool ok_last[3];
      for (int a = 0; a < 3; ++a) {
        Key nk = k;
        if (a == 0) nk.x += 1; else if (a == 1) nk.y += 1; else nk.z += 1;
        const Block<R, Sto>* nb = find(nk);
        ok_last[a] = nb != nullptr;
        h_last[a] = nb ? s + ((int64_t)1 << nb->level) : 0;
      }
      for (int iz = 0; iz < nl; ++iz)
        for (int iy = 0; iy < nl; ++iy)
          for (int ix = 0; ix < nl; ++ix) {
            const int i[3] = {ix, iy, iz};
            int64_t c[3], h[3];
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
              c[a] = K[a] * bu + (2 * i[a] + 1) * s;
              if (i[a] < nl - 1) h[a] = 2 * s;
              else { h[a] = h_last[a]; ok = ok && ok_last[a]; }
            }
            if (!ok) continue;
            R F[8];
            int64_t P[8][3];
            int cs = 0;
            for (int o = 0; o < 8 && ok; ++o) {
              for (int a = 0; a < 3; ++a) P[o][a] = c[a] + ((o >> a) & 1) * h[a];
              ok = mc_value(P[o], &F[o]);
              if (ok && F[o] < (R)0) cs |= 1 << o;
            }
            if (!ok) continue;
            for (int t = 0; t < tab.n_tris[cs]; ++t)
              for (int q = 0; q < 3; ++q) {
                const int e = tab.edges[cs][3 * t + q];
                const int c0 = tab.edge_corner[e][0], c1 = tab.edge_corner[e][1];
                const R f = F[c0] / (F[c0] - F[c1]);
                for (int a = 0; a < 3; ++a) {
                  const R pa = (R)P[c0][a] * unit, pb = (R)P[c1][a] * unit;
                  tris.push_back((float)(pa + f * (pb - pa)));
                }
              }
          }
    }
  }

  // ---- read-out, sorted by key (x, then y, then z)
  std::vector<Key> sorted_keys() const {
    std::vector<Key> ks;
    ks.reserve(blocks.size());
    for (auto& kv : blocks) ks.push_back(kv.first);
    std::sort(ks.begin(), ks.end());
    return ks;
  }

  int64_t count_blocks(int64_t* n_voxels) override {
    int64_t nv = 0;
    for (auto& kv : blocks) nv += (int64_t)kv.second.W.size();
    if (n_voxels) *n_voxels = nv;
    return (int64_t)blocks.size();
  }

  int extract(int32_t* keys, uint8_t* levels, int64_t* offsets, double* D, double* W, double* S2,
              double* C) override {
    std::vector<Key> ks = sorted_keys();
    int64_t off = 0;
    for (size_t i = 0; i < ks.size(); ++i) {
      const Block<R, Sto>& b = blocks.at(ks[i]);
      keys[3 * i] = (int32_t)ks[i].x;
      keys[3 * i + 1] = (int32_t)ks[i].y;
      keys[3 * i + 2] = (int32_t)ks[i].z;
      levels[i] = (uint8_t)b.level;
      offsets[i] = off;
      for (size_t j = 0; j < b.W.size(); ++j) {
        D[off + j] = (double)Store<Sto>::get(b.D[j]);
        W[off + j] = (double)b.W[j];
        S2[off + j] = (double)b.S2[j];
        if (C)
          for (int q = 0; q < 3; ++q) C[3 * (off + j) + q] = P.has_color ? (double)Store<Sto>::get(b.C[q][j]) : 0.0;
      }
      off += (int64_t)b.W.size();
    }
    offsets[ks.size()] = off;
    return 0;
  }

  int block_stats(int32_t* keys, uint8_t* levels, double* vbar, int64_t* n_obs, int64_t* sum_w) override {
    std::vector<Key> ks = sorted_keys();
    for (size_t i = 0; i < ks.size(); ++i) {
      const Block<R, Sto>& b = blocks.at(ks[i]);
      BStat s = stats(b);
      keys[3 * i] = (int32_t)ks[i].x;
      keys[3 * i + 1] = (int32_t)ks[i].y;
      keys[3 * i + 2] = (int32_t)ks[i].z;
      levels[i] = (uint8_t)b.level;
      vbar[i] = s.vbar;
      n_obs[i] = s.n_obs;
      sum_w[i] = s.sum_w;
    }
    return 0;
  }

  // ---- test hook: load one block payload, apply merge (dir = +1) or split (dir = -1), read it back
  int resample(int level, int dir, const double* D, const double* W, const double* S2, const double* C, double* oD,
               double* oW, double* oS2, double* oC) {
    if (level < 0 || level >= L || (dir > 0 && level >= L - 1) || (dir < 0 && level == 0)) return -1;
    Block<R, Sto> b;
    b.level = level;
    b.resize(n[level], P.has_color != 0);
    for (size_t i = 0; i < b.W.size(); ++i) {
      b.D[i] = Store<Sto>::put((R)D[i]);
      b.W[i] = (R)W[i];
      b.S2[i] = (R)S2[i];
      if (P.has_color)
        for (int q = 0; q < 3; ++q) b.C[q][i] = Store<Sto>::put((R)C[3 * i + q]);
    }
    if (dir > 0) merge(b); else split(b);
    for (size_t i = 0; i < b.W.size(); ++i) {
      oD[i] = (double)Store<Sto>::get(b.D[i]);
      oW[i] = (double)b.W[i];
      oS2[i] = (double)b.S2[i];
      if (oC)
        for (int q = 0; q < 3; ++q) oC[3 * i + q] = P.has_color ? (double)Store<Sto>::get(b.C[q][i]) : 0.0;
    }
    return 0;
  }
};

}  // namespace

// ------------------------------------------------------------------------------------------------ C interface

extern "C" {

void* orc_create(const orc_params* p) {
  if (!p || p->n_levels < 1 || p->n_levels > kMaxLevels || !(p->base_voxel > 0) || !(p->truncation > 0)) return nullptr;
  if (p->precision == 1) return new Map<double, double>(*p);
  if (p->fp16) return new Map<float, _Float16>(*p);
  return new Map<float, float>(*p);
}

void orc_destroy(void* h) { delete (MapBase*)h; }

int orc_integrate_depth(void* h, const orc_pinhole* K, const double* T_wc, const float* depth, const uint8_t* rgb,
                        orc_frame_stats* st) {
  return ((MapBase*)h)->integrate_depth(K, T_wc, depth, rgb, st);
}

int orc_integrate_points(void* h, const double* T_ws, const float* xyz, int64_t n, orc_frame_stats* st) {
  return ((MapBase*)h)->integrate_points(T_ws, xyz, n, st);
}

int orc_raycast(void* h, const orc_pinhole* K, const double* T_wc, float* depth_out, float* normal_out,
                uint8_t* rgb_out) {
  return ((MapBase*)h)->raycast(K, T_wc, depth_out, normal_out, rgb_out);
}

// the same for the listed pixels only (index v * width + u); outputs per listed pixel
int orc_raycast_pixels(void* h, const orc_pinhole* K, const double* T_wc, int64_t n, const int64_t* pix,
                       float* depth_out, float* normal_out, uint8_t* rgb_out) {
  return ((MapBase*)h)->raycast_pixels(K, T_wc, n, pix, depth_out, normal_out, rgb_out);
}

// test hook: the raycast's field at n world points (xyz, 3 doubles each; valid = 0 where it does not exist), and the
// unit normal and colour the raycast reports for a hit there (zeros where it reports none); outputs may be NULL
void orc_probe_points(void* h, int64_t n, const double* xyz, double* F, int8_t* valid, float* normal,
                      uint8_t* rgb) {
  ((MapBase*)h)->probe_points(n, xyz, F, valid, normal, rgb);
}

int orc_set_block(void* h, const int32_t* key, int level, const double* D, const double* W, const double* S2,
                  const double* C) {
  return ((MapBase*)h)->set_block(key, level, D, W, S2, C);
}

// capacity-driven streaming (fraction 0 disables); max_blocks[3] = pool capacity per level
void orc_set_streaming(void* h, float fraction, float radius, const int64_t* max_blocks) {
  ((MapBase*)h)->set_streaming(fraction, radius, max_blocks);
}
int64_t orc_archived(void* h) { return ((MapBase*)h)->archived(); }

// Extract the mesh; returns the triangle count. out (9 floats per triangle) may be NULL or smaller (cap triangles):
// the extraction is kept and later calls with out != NULL and extract == 0 copy it.
int64_t orc_extract_mesh(void* h, int extract, float* out, int64_t cap) {
  MapBase* m = (MapBase*)h;
  if (extract) {
    m->mesh.clear();
    m->extract_mesh(m->mesh);
  }
  const int64_t nt = (int64_t)(m->mesh.size() / 9);
  if (out)
    for (int64_t i = 0; i < 9 * std::min(nt, cap); ++i) out[i] = m->mesh[(size_t)i];
  return nt;
}

// Vertex collapse (Sec. 3.4, a reading): the vertices of a triangle soup are clustered on a grid of spacing delta
// (cluster of p = floor(p_a * (1 / delta)) per axis, in float); every cluster becomes one vertex, its lexicographically
// smallest member (x, then y, then z), numbered in ascending cluster order (x, then y, then z); triangles are
// re-indexed and those with two equal indices dropped, in soup order. Returns the vertex count; faces -> *n_faces.
int64_t orc_weld_mesh(const float* tris, int64_t n_tris, float delta, float* verts_out, int64_t cap_verts,
                      int32_t* faces_out, int64_t cap_faces, int64_t* n_faces) {
  const float inv = 1.0f / delta;
  std::map<std::array<int64_t, 3>, std::array<float, 3>> cl;
  std::vector<std::array<int64_t, 3>> key((size_t)(3 * n_tris));
  for (int64_t v = 0; v < 3 * n_tris; ++v) {
    const float* p = tris + 3 * v;
    std::array<int64_t, 3> k;
    for (int a = 0; a < 3; ++a) k[a] = (int64_t)std::floor(p[a] * inv);
    key[(size_t)v] = k;
    auto it = cl.find(k);
    const std::array<float, 3> q{p[0], p[1], p[2]};
    if (it == cl.end()) cl.emplace(k, q);
    else if (q < it->second) it->second = q;
  }
  std::map<std::array<int64_t, 3>, int32_t> index;
  int32_t nv = 0;
  for (auto& kv : cl) {
    if (verts_out && nv < cap_verts)
      for (int a = 0; a < 3; ++a) verts_out[3 * nv + a] = kv.second[a];
    index[kv.first] = nv++;
  }
  int64_t nf = 0;
  for (int64_t t = 0; t < n_tris; ++t) {
    const int32_t i0 = index[key[(size_t)(3 * t)]], i1 = index[key[(size_t)(3 * t + 1)]],
                  i2 = index[key[(size_t)(3 * t + 2)]];
    if (i0 == i1 || i1 == i2 || i0 == i2) continue;
    if (faces_out && nf < cap_faces) {
      faces_out[3 * nf] = i0;
      faces_out[3 * nf + 1] = i1;
      faces_out[3 * nf + 2] = i2;
    }
    ++nf;
  }
  *n_faces = nf;
  return nv;
}

// the case table (test hook): n_tris[256], edges[256 * 36], edge corners[24]
void orc_mc_table(int* n_tris, int8_t* edges, int8_t* edge_corner) {
  static const McTable t;
  for (int c = 0; c < 256; ++c) {
    n_tris[c] = t.n_tris[c];
    for (int i = 0; i < 36; ++i) edges[36 * c + i] = t.edges[c][i];
  }
  for (int e = 0; e < 12; ++e) {
    edge_corner[2 * e] = t.edge_corner[e][0];
    edge_corner[2 * e + 1] = t.edge_corner[e][1];
  }
}

int64_t orc_count_blocks(void* h, int64_t* n_voxels) { return ((MapBase*)h)->count_blocks(n_voxels); }

int orc_extract(void* h, int32_t* keys, uint8_t* levels, int64_t* offsets, double* D, double* W, double* S2,
                double* C) {
  return ((MapBase*)h)->extract(keys, levels, offsets, D, W, S2, C);
}

int orc_block_stats(void* h, int32_t* keys, uint8_t* levels, double* vbar, int64_t* n_obs, int64_t* sum_w) {
  return ((MapBase*)h)->block_stats(keys, levels, vbar, n_obs, sum_w);
}

// Geometry helpers exposed for the pin tests: cells of the closed fixed-point segment A -> B with cell edge U.
// mode 0 = bounding-box test of every cell, mode 1 = ordered walk. Returns the count (cells written up to cap).
int64_t orc_segment_cells(const int64_t* A, const int64_t* B, int64_t U, int mode, int64_t* out, int64_t cap) {
  std::vector<Key> c = mode == 0 ? cells_bruteforce(A, B, U) : cells_dda(A, B, U);
  for (size_t i = 0; i < c.size() && (int64_t)i < cap; ++i) {
    out[3 * i] = c[i].x;
    out[3 * i + 1] = c[i].y;
    out[3 * i + 2] = c[i].z;
  }
  return (int64_t)c.size();
}

float orc_half_round(float x) { return half_round(x); }

// Learned level predictor: weights (MRH-packed BF16 bits, 5443 values) or null to turn it off.
void orc_set_predictor(void* h, const uint16_t* w, int64_t n) {
  MapBase* m = (MapBase*)h;
  if (w) m->pred_w.assign(w, w + n);
  else m->pred_w.clear();
}

void orc_set_capture(void* h, int on) {
  MapBase* m = (MapBase*)h;
  m->capture = on != 0;
  m->cap_keys.clear();
  m->cap_feat.clear();
}

// Captured records in capture order; returns the count (records written up to cap).
int64_t orc_get_features(void* h, int32_t* keys, float* feats, int64_t cap) {
  MapBase* m = (MapBase*)h;
  const int64_t n = (int64_t)m->cap_keys.size();
  for (int64_t i = 0; i < n && i < cap; ++i) {
    keys[3 * i] = (int32_t)m->cap_keys[i].x;
    keys[3 * i + 1] = (int32_t)m->cap_keys[i].y;
    keys[3 * i + 2] = (int32_t)m->cap_keys[i].z;
    for (int q = 0; q < 16; ++q) feats[16 * i + q] = m->cap_feat[16 * i + q];
  }
  return n;
}

// Test hook: the merge (dir = +1) or split (dir = -1) payload rule applied to one block of the given level.
int orc_resample_block(void* h, int level, int dir, const double* D, const double* W, const double* S2,
                       const double* C, double* oD, double* oW, double* oS2, double* oC) {
  return ((MapBase*)h)->resample(level, dir, D, W, S2, C, oD, oW, oS2, oC);
}

}  // extern "C"
