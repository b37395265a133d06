// CPU reference build of the BVH -- TEST INFRASTRUCTURE ONLY, used to check
// the GPU build bit for bit.  Written independently of the CUDA code; the two
// agree because both follow the same published algorithms on the same float32
// inputs:
//   centroid  c = ((v0 + v1) + v2) / 3            (float32, no contraction)
//   quantise  q = trunc(((c - lo) / (hi - lo)) * 1024), clamped to [0, 1023]
//   Morton    interleave(qx, qy, qz) (x highest), key = morton << 32 | id
//   sort keys ascending (leaf slot i = i-th key)
//   PLOC (Meister & Bittner, IEEE TVCG 2018) over the sorted leaves: every
//   cluster's nearest neighbour within +-8 positions by least half surface
//   area ((dx*dy + dy*dz) + dz*dx in float32) of the merged box, ties to the
//   lower position; mutual pairs merge into a new node numbered
//   (n-2) - (order of creation, positions ascending within a round), the
//   clusters are compacted in order, until one remains (the root, node 0);
//   child reference = node index, or slot | 0x80000000 for a leaf;
//   child boxes = exact float min/max.
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
  auto merged = [](const Box& a, const Box& b) {
    Box r;
    for (int k = 0; k < 3; ++k) {
      r.lo[k] = std::min(a.lo[k], b.lo[k]);
      r.hi[k] = std::max(a.hi[k], b.hi[k]);
    }
    return r;
  };
  auto half_area = [](const Box& b) {
    volatile float dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    volatile float p = dx * dy, q = dy * dz, r = dz * dx;
    volatile float s1 = p + q;
    volatile float s2 = s1 + r;
    return (float)s2;
  };
  std::vector<Box> box(n);
  std::vector<int> ref(n);
  for (int i = 0; i < n; ++i) {
    box[i] = leaf_box(i);
    ref[i] = (int)(0x80000000u | (uint32_t)i);
  }
  const int R = 8;
  int created = 0;
  while (box.size() > 1) {
    const int m = (int)box.size();
    std::vector<int> nn(m);
    for (int i = 0; i < m; ++i) {
      int best = -1;
      float ba = 3.4e38f;
      for (int j = std::max(0, i - R); j <= std::min(m - 1, i + R); ++j) {
        if (j == i) continue;
        float a = half_area(merged(box[i], box[j]));
        if (a < ba || (a == ba && j < best)) {
          ba = a;
          best = j;
        }
      }
      nn[i] = best;
    }
    std::vector<Box> nb;
    std::vector<int> nr;
    for (int i = 0; i < m; ++i) {
      const int j = nn[i];
      const bool mutual = j >= 0 && nn[j] == i;
      if (mutual && j < i) continue;  // absorbed by its lower partner
      if (mutual) {
        const int x = (n - 2) - created++;
        lref[x] = ref[i];
        rref[x] = ref[j];
        child_box[2 * x] = box[i];
        child_box[2 * x + 1] = box[j];
        nb.push_back(merged(box[i], box[j]));
        nr.push_back(x);
      } else {
        nb.push_back(box[i]);
        nr.push_back(ref[i]);
      }
    }
    box.swap(nb);
    ref.swap(nr);
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
