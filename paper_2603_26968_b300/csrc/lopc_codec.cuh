// lopc_codec.cuh -- block-cooperative lossless stages on shared memory (Sec. III-C):
// BIT_w bit-plane transposes by warp butterflies (several groups of words per
// butterfly when the words reach few planes), and RZE_g (repeated zero elimination
// with a twice repeat-eliminated bitmap) as word-level encode/decode, plus 16-byte
// copies between a staged record and global memory.
#pragma once
#include "lopc_device.cuh"

namespace lopc {

// ------------------------------------------------------------- BIT_w stage

// 32 x 32 bit-matrix transpose across a warp: lane r holds row r (bit c = column
// c) on entry and column r on exit.  Five butterfly stages swap the off-diagonal
// s x s blocks between lanes r and r ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

// Bytes of a plane buffer (n32 / 32 words per plane, L bytes in all) that hold its
// first P planes, rounded up to 64 bytes (whole level-0 bitmap bytes of every RZE
// unit size used here) and clipped to L: where the coder can stop reading when the
// planes above P are zero.
__device__ __forceinline__ uint32_t plane_bytes_of(int n32, int P, uint32_t L) {
  const uint32_t b = ((uint32_t)P * (uint32_t)n32 / 8u + 63u) & ~63u;  // P planes of n32/32 words
  return b < L ? b : L;
}

// Planes a word OR-reduction `orw` reaches (the planes above are zero).
__device__ __forceinline__ int planes_of(uint64_t orw) { return orw ? 64 - __clzll((long long)orw) : 0; }

// After a partial rze_decode into `buf` (its first lw bytes, a multiple of 16,
// written): zeroes bytes [lw, end), 16 bytes a store (all threads; ends with a
// barrier).  `end` is a multiple of 16: the end of the planes a transpose will read.
template <int NT>
__device__ __forceinline__ void zero_after_decode(uint8_t* buf, uint32_t lw, uint32_t end) {
  uint4* b = reinterpret_cast<uint4*>(buf);
  for (uint32_t i = lw / 16u + threadIdx.x; i < end / 16u; i += NT) b[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
}

// Bit-plane transpose of n32 words (a multiple of 32): plane k (k = 0 least
// significant) is n32/32 u32 words, bit j of word g being bit k of word 32g+j.
// `word(i)` supplies input word i (zero for padding).  One warp per group of 32
// words; with a plane length that is a multiple of 4 a warp takes four groups at a
// time and each lane stores its four plane words in one 16-byte access (the lanes'
// words lie a plane apart, on the same banks, so this cuts the conflicts by four).
// Returns the OR of the words this thread transposed (the block-wide OR tells how
// many planes can be non-zero).
template <int NT, int W, typename WordFn>
__device__ __forceinline__ uint64_t bit_transpose(int n32, WordFn word, uint32_t* planes) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = n32 >> 5;
  uint64_t orw = 0;
  if ((G & 3) == 0) {
    for (int g = 4 * wid; g < G; g += 4 * (NT / 32)) {
      uint32_t lo[4], hi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint64_t v = word(32 * (g + u) + lane);
        orw |= v;
        lo[u] = warp_transpose32((uint32_t)v);
        hi[u] = W == 8 ? warp_transpose32((uint32_t)(v >> 32)) : 0u;
      }
      *reinterpret_cast<uint4*>(&planes[lane * G + g]) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      if (W == 8) *reinterpret_cast<uint4*>(&planes[(32 + lane) * G + g]) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    }
    return orw;
  }
  for (int g = wid; g < G; g += NT / 32) {
    const uint64_t v = word(32 * g + lane);
    orw |= v;
    planes[lane * G + g] = warp_transpose32((uint32_t)v);
    if (W == 8) planes[(32 + lane) * G + g] = warp_transpose32((uint32_t)(v >> 32));
  }
  return orw;
}

// Block-wide OR of each thread's `v` into *dst (zeroed beforehand and read after the
// caller's next barrier).
__device__ __forceinline__ void block_or_into(uint64_t v, unsigned long long* dst) {
  const uint64_t o = ((uint64_t)__reduce_or_sync(0xffffffffu, (unsigned)(v >> 32)) << 32) |
                     __reduce_or_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && o) atomicOr(dst, (unsigned long long)o);
}

// Packed transposes for words whose bits from P on are zero (P <= P2 = 2^LG <= 32).
// One 32 x 32 warp transpose then carries Q = 32 / P2 groups of 32 words: row
// j * P2 + k is plane k of group j, and column c holds the low P2 bits of word c of
// group j in bits [j P2, (j + 1) P2).  The planes are the same as bit_transpose's;
// planes [P2, W*8) are not written (they are zero), planes [P, P2) are written as zero.
template <int LG, int NT, typename WordFn>
__device__ __forceinline__ void transpose_packed(int G, WordFn word, uint32_t* planes) {
  constexpr int P2 = 1 << LG, Q = 32 >> LG;
  constexpr uint32_t MASK = P2 == 32 ? 0xffffffffu : (1u << P2) - 1u;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = lane >> LG, k = lane & (P2 - 1);
  for (int go = wid * Q; go < G; go += (NT / 32) * Q) {
    uint32_t v = 0;
#pragma unroll
    for (int jj = 0; jj < Q; ++jj)
      if (go + jj < G) v |= ((uint32_t)word(32 * (go + jj) + lane) & MASK) << (jj * P2);
    const uint32_t r = warp_transpose32(v);
    if (go + j < G) planes[k * G + go + j] = r;
  }
}

// Inverse of transpose_packed: reads planes [0, P) only.
template <int LG, int NT, typename EmitFn>
__device__ __forceinline__ void untranspose_packed(int G, const uint32_t* planes, int P, EmitFn emit) {
  constexpr int P2 = 1 << LG, Q = 32 >> LG;
  constexpr uint32_t MASK = P2 == 32 ? 0xffffffffu : (1u << P2) - 1u;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = lane >> LG, k = lane & (P2 - 1);
  for (int go = wid * Q; go < G; go += (NT / 32) * Q) {
    const int g = go + j;
    const uint32_t r = warp_transpose32(k < P && g < G ? planes[k * G + g] : 0u);
    // one copy of emit per variant: it is inlined, and unrolled copies of every packing
    // width overflow the instruction cache
#pragma unroll 1
    for (int jj = 0; jj < Q; ++jj)
      if (go + jj < G) emit(32 * (go + jj) + lane, (uint64_t)((r >> (jj * P2)) & MASK));
  }
}

// Whether the packed transposes serve a chunk of n32 words whose planes from P on are
// zero: P <= 16 (at least two groups per transpose), or P <= 32 for 64-bit words
// (one transpose instead of two), and whole 64-byte planes, so that the coder's
// plane_bytes_of(n32, P) ends on a plane the transpose wrote.
template <int W>
__device__ __forceinline__ bool packed_ok(int n32, int P) {
  return (n32 & 511) == 0 && (P <= 16 || (W == 8 && P <= 32));
}

// log2 of the packing width for P planes: 4 planes at least (eight groups).
__device__ __forceinline__ int packed_lg(int P) { return P <= 4 ? 2 : 32 - __clz(P - 1); }

// bit_transpose of words whose planes from P on are zero (the caller knows P, e.g.
// from an OR of the words): packed when packed_ok, else the plain transpose.
template <int NT, int W, typename WordFn>
__device__ __forceinline__ void bit_transpose_planes(int n32, int P, WordFn word, uint32_t* planes) {
  if (!packed_ok<W>(n32, P)) {
    (void)bit_transpose<NT, W>(n32, word, planes);
    return;
  }
  const int G = n32 >> 5;
  switch (packed_lg(P)) {
    case 2: transpose_packed<2, NT>(G, word, planes); break;
    case 3: transpose_packed<3, NT>(G, word, planes); break;
    case 4: transpose_packed<4, NT>(G, word, planes); break;
    default: transpose_packed<5, NT>(G, word, planes); break;
  }
}

// Inverse of bit_transpose: `emit(i, word)` receives word i of the n32.  Only planes
// [0, P) are read; the others are taken as zero.
template <int NT, int W, typename EmitFn>
__device__ __forceinline__ void bit_untranspose(int n32, const uint32_t* planes, EmitFn emit, int P = 8 * W) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = n32 >> 5;
  if (packed_ok<W>(n32, P)) {
    switch (packed_lg(P)) {
      case 2: untranspose_packed<2, NT>(G, planes, P, emit); break;
      case 3: untranspose_packed<3, NT>(G, planes, P, emit); break;
      case 4: untranspose_packed<4, NT>(G, planes, P, emit); break;
      default: untranspose_packed<5, NT>(G, planes, P, emit); break;
    }
    return;
  }
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  if ((G & 3) == 0) {
    for (int g = 4 * wid; g < G; g += 4 * (NT / 32)) {
      const uint4 a = lane < P ? *reinterpret_cast<const uint4*>(&planes[lane * G + g]) : z;
      uint4 b = z;
      if (W == 8 && 32 + lane < P) b = *reinterpret_cast<const uint4*>(&planes[(32 + lane) * G + g]);
      const uint32_t la[4] = {a.x, a.y, a.z, a.w}, lb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t lo = warp_transpose32(la[u]);
        const uint32_t hi = W == 8 ? warp_transpose32(lb[u]) : 0u;
        emit(32 * (g + u) + lane, (uint64_t)lo | ((uint64_t)hi << 32));
      }
    }
    return;
  }
  for (int g = wid; g < G; g += NT / 32) {
    const uint32_t lo = warp_transpose32(lane < P ? planes[lane * G + g] : 0u);
    const uint32_t hi = W == 8 ? warp_transpose32(32 + lane < P ? planes[(32 + lane) * G + g] : 0u) : 0u;
    emit(32 * g + lane, (uint64_t)lo | ((uint64_t)hi << 32));
  }
}

// Planes of a buffer of n32-word planes that a partial RZE decode of lw bytes can have
// made non-zero (all planes from there on are zero), and the end of the bytes that must
// be zeroed after the decode for bit_untranspose(..., P): the rest of plane P - 1,
// rounded up to 16 and clipped to L.
__device__ __forceinline__ int planes_in(uint32_t lw, int n32) {
  const uint32_t pb = (uint32_t)n32 / 8u;  // bytes of a plane
  return (int)((lw + pb - 1u) / pb);
}
__device__ __forceinline__ uint32_t planes_zero_end(int P, int n32, uint32_t L) {
  const uint32_t e = ((uint32_t)P * ((uint32_t)n32 / 8u) + 15u) & ~15u;
  return e < L ? e : L;
}

// ------------------------------------------------------------- RZE_g stage

// Scratch of one RZE pass over at most Lmax bytes.
struct RzeWork {
  uint8_t* m0;    // level-0 bitmap, >= Lmax/8 + 8 bytes
  uint8_t* m1;    // level-1 bitmap, >= Lmax/64 + 8 bytes
  uint8_t* m2;    // level-2 bitmap, >= Lmax/512 + 8 bytes
  uint32_t* pre;  // prefix counts of m1 words, >= Lmax/256 + 8 words
  uint32_t* tmp;  // scan slots, >= 40 words
  static constexpr size_t a16(size_t v) { return (v + 15) & ~(size_t)15; }
  static constexpr size_t bytes(uint32_t Lmax) {
    return a16(Lmax / 8 + 16) + a16(Lmax / 64 + 16) + a16(Lmax / 512 + 16) + ((size_t)Lmax / 256 + 8) * 4 + 40 * 4;
  }
};

// Carves the scratch out of `base` (16-byte aligned); every part is 16-byte aligned.
__device__ __forceinline__ RzeWork rze_work_at(uint8_t* base, uint32_t Lmax) {
  RzeWork w;
  w.m0 = base;
  w.m1 = w.m0 + RzeWork::a16(Lmax / 8 + 16);
  w.m2 = w.m1 + RzeWork::a16(Lmax / 64 + 16);
  w.pre = reinterpret_cast<uint32_t*>(w.m2 + RzeWork::a16(Lmax / 512 + 16));
  w.tmp = w.pre + Lmax / 256 + 8;
  return w;
}

__device__ __forceinline__ uint32_t ceil8(uint32_t n) { return (n + 7u) >> 3; }

// Non-zero flags of the 4 bytes of w as a nibble (bit i = byte i non-zero).
__device__ __forceinline__ uint32_t nz_nibble(uint32_t w) {
  const uint32_t h = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
  return (((h >> 7) * 0x204081u) >> 21) & 0xFu;
}

// Level-0 bitmap byte j: bit b set when unit 8j+b (of U units of G bytes) is non-zero.
template <int G>
__device__ __forceinline__ uint32_t level0_byte(const uint8_t* in, uint32_t U, uint32_t j) {
  const uint32_t u0 = 8 * j;
  if (u0 + 8 <= U) {
    if (G == 1) {
      const uint2 v = *reinterpret_cast<const uint2*>(in + u0);
      return nz_nibble(v.x) | (nz_nibble(v.y) << 4);
    } else if (G == 4) {
      const uint4 a = *reinterpret_cast<const uint4*>(in + 4 * u0);
      const uint4 b = *reinterpret_cast<const uint4*>(in + 4 * u0 + 16);
      return (a.x != 0) | ((a.y != 0) << 1) | ((a.z != 0) << 2) | ((a.w != 0) << 3) | ((b.x != 0) << 4) |
             ((b.y != 0) << 5) | ((b.z != 0) << 6) | ((b.w != 0) << 7);
    } else {
      uint32_t r = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint2 v = *reinterpret_cast<const uint2*>(in + 8 * (u0 + k));
        r |= (uint32_t)((v.x | v.y) != 0) << k;
      }
      return r;
    }
  }
  uint32_t r = 0;
  for (uint32_t k = 0; k < 8 && u0 + k < U; ++k) {
    uint32_t nz = 0;
    for (int b = 0; b < G; ++b) nz |= in[(u0 + k) * G + b];
    r |= (nz != 0) << k;
  }
  return r;
}

// Warp-level exclusive scan of v; *total gets the warp's sum.
__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t v, uint32_t* total) {
  const int lane = threadIdx.x & 31;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// Level-0 bitmap bytes are split into one contiguous range per warp; within a
// range, lane l takes bytes 32*step + l, so a warp touches consecutive memory.
template <int NT>
struct WarpRange {
  uint32_t a, b;  // bitmap bytes [a, b) of this warp
  __device__ WarpRange(uint32_t l0) {
    constexpr int NW = NT / 32;
    const uint32_t cw = ((l0 + NW - 1) / NW + 31) & ~31u;
    a = min(l0, (uint32_t)(threadIdx.x >> 5) * cw);
    b = min(l0, a + cw);
  }
};

// Exclusive block scan of three counters at once, with one barrier: a[j] receives the
// sum of v[j] over the threads before this one, tot[j] the block's sum.  `tmp` holds
// 3 * NT/32 words and must not be reused before the next barrier.
template <int NT>
__device__ __forceinline__ void block_exclusive_scan3(const uint32_t v[3], uint32_t* tmp, uint32_t a[3],
                                                      uint32_t tot[3]) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x[j], o);
      if (lane >= o) x[j] += y;
    }
  }
  if (lane == 31)
    for (int j = 0; j < 3; ++j) tmp[3 * wid + j] = x[j];
  __syncthreads();
  for (int j = 0; j < 3; ++j) {
    uint32_t base = 0, all = 0;
    for (int k = 0; k < NW; ++k) {
      const uint32_t t = tmp[3 * k + j];
      base += k < wid ? t : 0u;
      all += t;
    }
    a[j] = base + x[j] - v[j];
    tot[j] = all;
  }
}

// RZE_g encode of `in` (L bytes, shared memory, 16-byte aligned) into `out` (shared
// memory): [level-2 bitmap][level-1 kept][level-0 kept][non-zero units].  Nothing is
// written when the result would not be shorter than `limit`.  Returns its length.
// Bytes of `in` from Lnz on are taken as zero and not read (Lnz: a multiple of 8 G
// bytes, or >= L); the record is the same as for the whole input.
// Needs ceil(L/G/512) <= NT (true for the chunk sizes used here).
template <int NT, int G>
__device__ uint32_t rze_encode(const uint8_t* in, uint32_t L, uint8_t* out, uint32_t limit, const RzeWork& w,
                               uint32_t Lnz = 0xffffffffu) {
  const uint32_t U = L / G;
  const uint32_t l0 = ceil8(U), l1 = ceil8(l0), l2 = ceil8(l1);
  const uint32_t l0nz = Lnz >= L ? l0 : Lnz / (8u * G);  // level-0 bytes that can be non-zero
  const int t = threadIdx.x, lane = t & 31;
  const WarpRange<NT> wr(l0nz);
  auto m0at = [&](uint32_t j) -> uint32_t { return j < l0nz ? (uint32_t)w.m0[j] : 0u; };
  // level 0, warp-strided
  uint32_t c0 = 0;
  for (uint32_t j = wr.a + lane; j < wr.b; j += 32) {
    const uint32_t byte = level0_byte<G>(in, U, j);
    w.m0[j] = (uint8_t)byte;
    c0 += __popc(byte);
  }
  __syncthreads();
  // level 1: contiguous level-1 bytes per thread (few)
  const uint32_t per1 = (l1 + NT - 1) / NT;
  const uint32_t a1 = min(l1, (uint32_t)t * per1), b1 = min(l1, a1 + per1);
  uint32_t c1 = 0;
  for (uint32_t jj = a1; jj < b1; ++jj) {
    uint32_t byte = 0;
    if (8 * jj <= l0nz) {  // past the non-zero level-0 bytes nothing changes
      for (uint32_t b = 0; b < 8; ++b) {
        const uint32_t j = 8 * jj + b;
        if (j >= l0) break;
        const uint32_t prev = j ? m0at(j - 1) : 0u;
        if (m0at(j) != prev) byte |= 1u << b;
      }
    }
    w.m1[jj] = (uint8_t)byte;
    c1 += __popc(byte);
  }
  __syncthreads();  // level 1 complete
  // level 2: each thread owns one level-2 byte (8 level-1 bytes)
  uint32_t c2 = 0;
  if ((uint32_t)t < l2) {
    uint32_t byte = 0;
    for (uint32_t b = 0; b < 8; ++b) {
      const uint32_t j = 8 * t + b;
      if (j >= l1) break;
      const uint8_t prev = j ? w.m1[j - 1] : 0;
      if (w.m1[j] != prev) byte |= 1u << b;
    }
    w.m2[t] = (uint8_t)byte;
    c2 = __popc(byte);
  }
  // one scan: warps' payload bases, level-0 kept offsets, level-1 kept offsets
  uint32_t wtot;
  warp_exclusive_scan(c0, &wtot);
  const uint32_t sv3[3] = {lane == 0 ? wtot : 0u, c1, c2};
  uint32_t ex3[3], tot3[3];
  block_exclusive_scan3<NT>(sv3, w.tmp, ex3, tot3);
  const uint32_t warp_base = __shfl_sync(0xffffffffu, ex3[0], 0);
  const uint32_t k0_off = ex3[1], k1_off = ex3[2];
  const uint32_t np = tot3[0], nk0 = tot3[1], nk1 = tot3[2];
  const uint32_t total = l2 + nk1 + nk0 + np * G;
  if (total >= limit) return total;
  if ((uint32_t)t < l2) {
    out[t] = w.m2[t];
    uint32_t r = 0;
    for (uint32_t b = 0; b < 8; ++b)
      if ((w.m2[t] >> b) & 1u) out[l2 + k1_off + r++] = w.m1[8 * t + b];
  }
  {
    uint32_t r = 0;
    uint8_t* k0 = out + l2 + nk1 + k0_off;
    for (uint32_t jj = a1; jj < b1; ++jj) {
      uint32_t bits = w.m1[jj];
      while (bits) {
        const uint32_t j = 8 * jj + (__ffs(bits) - 1);
        bits &= bits - 1;
        k0[r++] = (uint8_t)m0at(j);
      }
    }
  }
  {
    uint8_t* pay = out + l2 + nk1 + nk0;
    uint32_t run = warp_base;
    for (uint32_t base = wr.a; base < wr.b; base += 32) {
      const uint32_t j = base + lane;
      const uint32_t bits = j < wr.b ? (uint32_t)w.m0[j] : 0u;
      uint32_t stot;
      uint32_t r = run + warp_exclusive_scan(__popc(bits), &stot);
      uint32_t bb = bits;
      while (bb) {
        const uint32_t u = 8 * j + (__ffs(bb) - 1);
        bb &= bb - 1;
#pragma unroll
        for (int b = 0; b < G; ++b) pay[r * G + b] = in[u * G + b];
        ++r;
      }
      run += stot;
    }
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ bool tail_clear(const uint8_t* bm, uint32_t nbits) {
  const uint32_t r = nbits & 7;
  return !r || (bm[nbits >> 3] >> r) == 0;
}

// RZE_g decode: `in` (in_len bytes, shared memory) -> `out` (L bytes, shared
// memory, 16-byte aligned).  Returns false for an inconsistent record.  With
// `written` null the whole output is written; otherwise only its first *written
// bytes (the bytes up to the last non-zero unit, rounded up to 64 and clipped to L),
// and every later byte of the output is zero.
template <int NT, int G>
__device__ bool rze_decode(const uint8_t* in, uint32_t in_len, uint32_t L, uint8_t* out, const RzeWork& w,
                           uint32_t* written = nullptr) {
  const uint32_t U = L / G;
  const uint32_t l0 = ceil8(U), l1 = ceil8(l0), l2 = ceil8(l1);
  const int t = threadIdx.x, lane = t & 31;
  if (in_len < l2) return false;  // uniform
  const uint8_t* m2 = in;
  // level-1 bitmap from level 2: warp 0 ranks the level-2 bytes (prefix popcounts,
  // 32 bytes per step), then every level-1 byte is one lookup
  if (t < 32) {
    uint32_t carry = 0;
    for (uint32_t base = 0; base < l2; base += 32) {
      const uint32_t i = base + t;
      const uint32_t c = i < l2 ? __popc((uint32_t)m2[i]) : 0u;
      uint32_t tot;
      const uint32_t ex = warp_exclusive_scan(c, &tot);
      if (i < l2) w.pre[i] = carry + ex;
      carry += tot;
    }
    if (t == 0) w.pre[l2] = carry;
  }
  __syncthreads();
  const uint32_t nk1 = w.pre[l2];
  if (!tail_clear(m2, l1) || l2 + nk1 > in_len) return false;  // uniform
  for (uint32_t j = t; j < ((l1 + 3) & ~3u); j += NT) {
    uint8_t v = 0;
    if (j < l1) {
      const uint32_t r = w.pre[j >> 3] + __popc((uint32_t)m2[j >> 3] & ((2u << (j & 7)) - 1u));
      v = r ? in[l2 + r - 1] : 0;
    }
    w.m1[j] = v;
  }
  __syncthreads();
  // prefix counts of level-1 words (warp 0); for a partial decode also the level-0
  // bytes that can be non-zero: m0 changes last at the last set bit jl of m1, to the
  // last kept level-0 byte, so m0 is zero from jl on when that byte is 0
  const uint32_t nw1 = (l1 + 3) >> 2;
  const uint32_t* m1w = reinterpret_cast<const uint32_t*>(w.m1);
  if (t < 32) {
    uint32_t carry = 0, last = 0;  // last: 1 + the highest set bit of m1 seen so far
    for (uint32_t base = 0; base < nw1; base += 32) {
      const uint32_t wi = base + t;
      const uint32_t mw = wi < nw1 ? m1w[wi] : 0u;
      const uint32_t c = __popc(mw);
      uint32_t tot;
      const uint32_t ex = warp_exclusive_scan(c, &tot);
      if (wi < nw1) w.pre[wi] = carry + ex;
      carry += tot;
      const uint32_t hi = __ballot_sync(0xffffffffu, mw != 0u);
      if (hi) {
        const int hl = 31 - __clz(hi);
        const uint32_t hw = __shfl_sync(0xffffffffu, mw, hl);
        last = 32 * (base + hl) + (32 - __clz(hw));
      }
    }
    if (t == 0) {
      w.pre[nw1] = carry;
      w.tmp[39] = last;
    }
  }
  __syncthreads();
  const uint32_t nk0 = w.pre[nw1];
  if (!tail_clear(w.m1, l0) || l2 + nk1 + nk0 > in_len) return false;  // uniform
  const uint8_t* k0 = in + l2 + nk1;
  uint32_t l0nz = l0;  // level-0 bytes that can be non-zero
  if (written) l0nz = nk0 == 0 ? 0u : (k0[nk0 - 1] != 0 ? l0 : min(l0, w.tmp[39] - 1u));
  for (uint32_t j = t; j < ((l0nz + 3) & ~3u); j += NT) {
    uint8_t v = 0;
    if (j < l0nz) {
      const uint32_t r = w.pre[j >> 5] + __popc(m1w[j >> 5] << (31 - (j & 31)));
      v = r ? k0[r - 1] : 0;
    }
    w.m0[j] = v;
  }
  __syncthreads();
  if (l0nz == l0 && !tail_clear(w.m0, U)) return false;  // uniform (a shorter m0 ends in zeros)
  // payload, warp-strided over the level-0 bytes
  const WarpRange<NT> wr(l0nz);
  uint32_t c0 = 0;
  for (uint32_t j = wr.a + lane; j < wr.b; j += 32) c0 += __popc((uint32_t)w.m0[j]);
  uint32_t wtot;
  warp_exclusive_scan(c0, &wtot);
  const uint32_t sv3[3] = {lane == 0 ? wtot : 0u, 0u, 0u};
  uint32_t ex3[3], tot3[3];
  block_exclusive_scan3<NT>(sv3, w.tmp, ex3, tot3);  // one barrier
  const uint32_t np = tot3[0];
  if ((uint64_t)l2 + nk1 + nk0 + (uint64_t)np * G != in_len) return false;  // uniform
  const uint8_t* pay = in + l2 + nk1 + nk0;
  uint32_t run = __shfl_sync(0xffffffffu, ex3[0], 0);
  for (uint32_t base = wr.a; base < wr.b; base += 32) {
    const uint32_t j = base + lane;
    const uint32_t bits = j < wr.b ? (uint32_t)w.m0[j] : 0u;
    uint32_t stot;
    uint32_t r = run + warp_exclusive_scan(__popc(bits), &stot);
    run += stot;
    if (j >= wr.b) continue;
    const uint32_t u0 = 8 * j;
    if (G == 1 && u0 + 8 <= U) {
      uint32_t lo = 0, hi = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        uint32_t v = 0;
        if ((bits >> b) & 1u) v = pay[r++];
        if (b < 4)
          lo |= v << (8 * b);
        else
          hi |= v << (8 * (b - 4));
      }
      *reinterpret_cast<uint2*>(out + u0) = make_uint2(lo, hi);
    } else {
      for (uint32_t b = 0; b < 8 && u0 + b < U; ++b) {
        if ((bits >> b) & 1u) {
#pragma unroll
          for (int k = 0; k < G; ++k) out[(u0 + b) * G + k] = pay[r * G + k];
          ++r;
        } else {
#pragma unroll
          for (int k = 0; k < G; ++k) out[(u0 + b) * G + k] = 0;
        }
      }
    }
  }
  if (written) {
    const uint32_t done = min(L, 8u * G * l0nz), lw = min(L, (done + 63u) & ~63u);
    for (uint32_t i = done + t; i < lw; i += NT) out[i] = 0;
    *written = lw;
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------- record copies

// Copies n bytes (rounded up to 16) between 16-byte aligned buffers.
template <int NT>
__device__ __forceinline__ void copy16(uint8_t* dst, const uint8_t* src, uint32_t n) {
  const uint32_t n16 = (n + 15) >> 4;
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (uint32_t i = threadIdx.x; i < n16; i += NT) d[i] = s[i];
}

// Zeroes bytes [n, pad16(n)) of a shared buffer (record padding).
template <int NT>
__device__ __forceinline__ void zero_tail16(uint8_t* buf, uint32_t n) {
  const uint32_t p = (n + 15) & ~15u;
  for (uint32_t i = n + threadIdx.x; i < p; i += NT) buf[i] = 0;
}

}  // namespace lopc
