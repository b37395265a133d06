// CPU reference build of a linear BVH (Karras, "Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees", HPG 2012) -- TEST
// INFRASTRUCTURE ONLY, used to check the GPU build bit for bit.  Written
// independently of the CUDA code; the two agree because both follow the same
// published algorithm on the same float32 inputs:
//   centroid  c = ((v0 + v1) + v2) / 3            (float32, no contraction)
//   quantise  q = trunc(((c - lo) / (hi - lo)) * 1024), clamped to [0, 1023]
//   Morton    interleave(qx, qy, qz) (x highest), key = morton << 32 | id
//   sort keys ascending; internal node i of n-1: range, split (Karras),
//   child reference = index, or index | 0x80000000 for a leaf;
//   child boxes = exact float min/max of the subtree's triangle vertices.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

uint32_t spread10(uint32_t v) {
  // move bit k of a 10-bit value to bit 3k
  uint32_t r = 0;
  for (int k = 0; k < 10; ++k) r |= ((v >> k) & 1u) << (3 * k);
  return r;
}

int common_prefix(const std::vector<uint64_t>& keys, int i, int j) {
  int n = (int)keys.size();
  if (j < 0 || j >= n) return -1;
  uint64_t x = keys[i] ^ keys[j];
  if (x == 0) return 64;
  int c = 0;
  while (!(x & (1ull << 63))) {
    x <<= 1;
    ++c;
  }
  return c;
}

struct Box {
  float lo[3], hi[3];
};

}  // namespace

extern "C" int oracle_lbvh_build(int n, const float* verts, uint64_t* keys_out, int32_t* children_out,
                                 float* boxes_out) {
  if (n <= 0) return 0;
  // centroid bounds
  std::vector<float> cen(3 * (size_t)n);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      volatile float s = verts[9 * i + a] + verts[9 * i + 3 + a];
      volatile float s2 = s + verts[9 * i + 6 + a];
      cen[3 * i + a] = s2 / 3.0f;
    }
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = cen[a];
    hi[a] = cen[a];
  }
  for (int i = 1; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], cen[3 * i + a]);
      hi[a] = std::max(hi[a], cen[3 * i + a]);
    }
  std::vector<uint64_t> keys(n);
  for (int i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      volatile float ext = hi[a] - lo[a];
      float t = 0.0f;
      if (ext > 0.0f) {
        volatile float num = cen[3 * i + a] - lo[a];
        t = num / ext;
      }
      volatile float sc = t * 1024.0f;
      int qi = (int)sc;
      q[a] = (uint32_t)std::min(1023, std::max(0, qi));
    }
    uint32_t m = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    keys[i] = ((uint64_t)m << 32) | (uint32_t)i;
  }
  std::sort(keys.begin(), keys.end());
  for (int i = 0; i < n; ++i) keys_out[i] = keys[i];
  if (n == 1) return 1;
  std::vector<int> lref(n - 1), rref(n - 1);
  for (int i = 0; i < n - 1; ++i) {
    int d = common_prefix(keys, i, i + 1) > common_prefix(keys, i, i - 1) ? 1 : -1;
    int dmin = common_prefix(keys, i, i - d);
    int lmax = 2;
    while (common_prefix(keys, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
      if (common_prefix(keys, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = common_prefix(keys, i, j);
    // binary search for the split: largest s with common prefix > dnode
    int s = 0;
    int t = l;
    while (t > 1) {
      t = (t + 1) / 2;
      if (common_prefix(keys, i, i + (s + t) * d) > dnode) s += t;
    }
    if (l == 1) {
      // single step: the search above never ran; the split is at i
      s = 0;
    }
    int gamma = i + s * d + std::min(d, 0);
    int first = std::min(i, j), last = std::max(i, j);
    lref[i] = (first == gamma) ? (int)(0x80000000u | (uint32_t)gamma) : gamma;
    rref[i] = (last == gamma + 1) ? (int)(0x80000000u | (uint32_t)(gamma + 1)) : gamma + 1;
  }
  // child boxes, bottom-up by recursion from the root (node 0)
  std::vector<Box> node_box(n - 1);
  std::vector<Box> child_box(2 * (size_t)(n - 1));
  auto leaf_box = [&](int slot) {
    int id = (int)(keys[slot] & 0xffffffffu);
    const float* v = verts + 9 * id;
    Box b;
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = std::min(std::min(v[a], v[3 + a]), v[6 + a]);
      b.hi[a] = std::max(std::max(v[a], v[3 + a]), v[6 + a]);
    }
    return b;
  };
  // iterative post-order
  std::vector<std::pair<int, int>> stack;
  stack.push_back({0, 0});
  while (!stack.empty()) {
    auto& top = stack.back();
    int node = top.first;
    if (top.second == 0) {
      top.second = 1;
      if (lref[node] >= 0) stack.push_back({lref[node], 0});
      if (rref[node] >= 0) stack.push_back({rref[node], 0});
      continue;
    }
    stack.pop_back();
    Box L = lref[node] < 0 ? leaf_box(lref[node] & 0x7fffffff) : node_box[lref[node]];
    Box R = rref[node] < 0 ? leaf_box(rref[node] & 0x7fffffff) : node_box[rref[node]];
    child_box[2 * node] = L;
    child_box[2 * node + 1] = R;
    Box U;
    for (int a = 0; a < 3; ++a) {
      U.lo[a] = std::min(L.lo[a], R.lo[a]);
      U.hi[a] = std::max(L.hi[a], R.hi[a]);
    }
    node_box[node] = U;
  }
  for (int i = 0; i < n - 1; ++i) {
    children_out[2 * i] = lref[i];
    children_out[2 * i + 1] = rref[i];
    const Box& L = child_box[2 * i];
    const Box& R = child_box[2 * i + 1];
    float* o = boxes_out + 12 * (size_t)i;
    for (int a = 0; a < 3; ++a) {
      o[a] = L.lo[a];
      o[3 + a] = L.hi[a];
      o[6 + a] = R.lo[a];
      o[9 + a] = R.hi[a];
    }
  }
  return n;
}
