// pp_host.cu -- C ABI of the GB300 ParPaRaw parser (declared in
// include/parparaw.h): table validation, scratch management, the init and
// finalize kernels, and the launch of the tile kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "pp_device.cuh"
#include "pp_launch.h"
#include "pp_parser.h"
#include "pp_types.h"


namespace pp {
namespace {

constexpr uint32_t kBlockInit = 256;
constexpr uint32_t kBlockFinal = 256;

// --------------------------------------------------------- init kernel ---
// Zeroes every job's look-back flags, fail / null bitmaps and bookkeeping.
__global__ void pp_init_kernel(const __grid_constant__ Launch L) {
  for (uint32_t j = blockIdx.y; j < L.njobs; j += gridDim.y) {
    const Job& J = L.jobs ? L.jobs[j] : L.job0;
    const Tables& TB = L.jobs ? L.tables[J.tables] : L.tables0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i < J.ntiles; i += stride) {
      J.st_state[i] = 0;
      J.st_rc[i] = 0;
    }
    const uint64_t nb = J.ntiles * TB.num_str;
    for (uint64_t i = i0; i < nb; i += stride) J.st_bytes[i] = 0;
    const uint64_t nbits = J.bit_words * (1 + static_cast<uint64_t>(TB.num_num));
    for (uint64_t i = i0; i < nbits; i += stride) {
      if (i < J.bit_words) J.fail_bits[i] = 0;
      else J.null_bits[i - J.bit_words] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Misc* M = J.misc;
      M->first_invalid = ~0ull;
      M->timeout = 0;
      M->done = 0;
      M->rows = 0;
      M->final_state = TB.start_state;
      M->last_record_end = 0;
      for (int k = 0; k < PP_MAX_STRING_COLUMNS; ++k) M->bytes_total[k] = 0;
      for (int k = 0; k < PP_MAX_COLUMNS; ++k) M->inf_rank[k] = 0;
      M->inf_min_fields = 0xFFFFFFFFu;
      M->inf_max_fields = 0;
      if (J.result != nullptr) J.result->n_rejected = 0;
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *L.work_counter = L.first_item;
}

__device__ __forceinline__ void put_bitmap_word(uint8_t* bm, uint64_t w, uint32_t bits, uint64_t nbytes) {
  for (int k = 0; k < 4; ++k) {
    const uint64_t b = 4 * w + k;
    if (b < nbytes) bm[b] = static_cast<uint8_t>(bits >> (8 * k));
  }
}

// ----------------------------------------------------- finalize kernel ---
// Turns the fail / null bitmaps into Arrow validity bitmaps and row_valid,
// counts rejected rows and writes the result of every job.
__global__ void pp_finalize_kernel(const __grid_constant__ Launch L) {
  __shared__ unsigned long long s_rej;
  for (uint32_t j = blockIdx.y; j < L.njobs; j += gridDim.y) {
    const Job& J = L.jobs ? L.jobs[j] : L.job0;
    const Tables& TB = L.jobs ? L.tables[J.tables] : L.tables0;
    const Col* cols = L.jobs ? (L.cols + J.col0) : L.cols0;
    const Misc& M = *J.misc;
    const bool ok_run = (J.ntiles == 0) || M.done;
    const int64_t R = ok_run ? M.rows : 0;
    const uint64_t rows_out = min(static_cast<uint64_t>(R), J.rows_cap);
    const uint64_t words = (rows_out + 31) / 32;
    const uint64_t nbytes = (rows_out + 7) / 8;
    if (threadIdx.x == 0) s_rej = 0;
    __syncthreads();
    unsigned long long rej = 0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t w = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < words; w += stride) {
      const uint32_t live = (w + 1 == words && (rows_out & 31)) ? ((1u << (rows_out & 31)) - 1u) : ~0u;
      const uint32_t fail = J.fail_bits[w] & live;
      const uint32_t ok = ~fail & live;
      rej += __popc(fail);
      put_bitmap_word(J.row_valid, w, ok, nbytes);
      for (uint32_t c = 0; c < TB.num_columns; ++c) {
        uint32_t bits = ok;
        if (TB.num_slot[c] != 0xFF) bits &= ~J.null_bits[TB.num_slot[c] * J.bit_words + w];
        if (cols[c].validity != nullptr) put_bitmap_word(cols[c].validity, w, bits, nbytes);
      }
    }
    for (int off = 16; off > 0; off >>= 1) rej += __shfl_xor_sync(0xffffffffu, rej, off);
    if ((threadIdx.x & 31) == 0 && rej) atomicAdd(&s_rej, rej);
    __syncthreads();
    if (threadIdx.x == 0 && s_rej) atomicAdd(reinterpret_cast<unsigned long long*>(&J.result->n_rejected), s_rej);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      pp_parse_result* res = J.result;
      int32_t status = PP_OK;
      bool cap = static_cast<uint64_t>(R) > J.rows_cap;
      for (uint32_t c = 0; c < TB.num_columns; ++c) {
        const uint32_t slot = TB.str_slot[c];
        const int64_t need = slot != 0xFF ? M.bytes_total[slot] : 0;
        res->values_bytes_needed[c] = need;
        if (slot != 0xFF) {
          cols[c].offsets[0] = 0;
          if (static_cast<uint64_t>(need) > cols[c].values_cap) cap = true;
        }
      }
      for (uint32_t c = TB.num_columns; c < PP_MAX_COLUMNS; ++c) res->values_bytes_needed[c] = 0;
      if (M.timeout || !ok_run) status = PP_E_TIMEOUT;
      else if (cap) status = PP_E_CAPACITY;
      else if (M.first_invalid != ~0ull) status = PP_E_INVALID_INPUT;
      else if (!TB.partial && !((TB.accept_mask >> M.final_state) & 1u)) status = PP_E_UNTERMINATED;
      res->status = status;
      res->final_state = M.final_state;
      res->rows = R;
      res->first_invalid_offset = M.first_invalid == ~0ull ? -1 : static_cast<int64_t>(M.first_invalid);
      res->consumed = TB.partial ? static_cast<int64_t>(M.last_record_end) : static_cast<int64_t>(J.len);
    }
    __syncthreads();
  }
}

// The inference result of the single job of an inference launch.
__global__ void pp_infer_finalize_kernel(const __grid_constant__ Launch L, pp_inference* out) {
  const Job& J = L.job0;
  const Tables& TB = L.tables0;
  const Misc& M = *J.misc;
  const int c = threadIdx.x;
  if (c < PP_MAX_COLUMNS) {
    const uint8_t of_rank[5] = {PP_TYPE_NONE, PP_INT32, PP_INT64, PP_FLOAT64, PP_STRING};
    out->type[c] = of_rank[min(M.inf_rank[c], 4u)];
  }
  if (c == 0) {
    const bool ok_run = (J.ntiles == 0) || M.done;
    int32_t status = PP_OK;
    if (M.timeout || !ok_run) status = PP_E_TIMEOUT;
    else if (M.first_invalid != ~0ull) status = PP_E_INVALID_INPUT;
    else if (!((TB.accept_mask >> M.final_state) & 1u)) status = PP_E_UNTERMINATED;
    out->status = status;
    out->records = ok_run ? M.rows : 0;
    out->min_fields = out->records > 0 && M.inf_min_fields != 0xFFFFFFFFu ? M.inf_min_fields : 0u;
    out->max_fields = out->records > 0 ? M.inf_max_fields : 0u;
    out->pad = 0;
    out->first_invalid_offset = M.first_invalid == ~0ull ? -1 : static_cast<int64_t>(M.first_invalid);
  }
}

// ------------------------------------------------------ device caches ---

struct KernelSlot {
  std::once_flag once;
  int blocks_per_sm = 0;
  cudaError_t err = cudaSuccess;
};

std::mutex g_mu;

ShapeInfo shape_for(int cfg) {
  switch (cfg) {
    case 1: return shape_info_tiny();
    case 2: return shape_info_small();
    case 3: return shape_info_mid();
    case 4: return shape_info_wide();
    case 5: return shape_info_m128();
    case 6: return shape_info_m128x6();
    case 7: return shape_info_s128();
    case 8: return shape_info_mid3();
    case 9: return shape_info_y96();
    case 10: return shape_info_t448();
    case 11: return shape_info_w48();
    case 12: return shape_info_big3();
    case 13: return shape_info_q384();
    case 14: return shape_info_q448();
    default: return shape_info_t448();
  }
}

struct DeviceProps {
  int sms = 0;
};

cudaError_t device_props(int dev, DeviceProps* out) {
  static std::unordered_map<int, DeviceProps> cache;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = cache.find(dev);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  DeviceProps p;
  cudaError_t e = cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cache[dev] = p;
  *out = p;
  return cudaSuccess;
}

// resident blocks per SM of one kernel on one device (sets the shared-memory
// attribute the first time)
cudaError_t kernel_occupancy(const void* kernel, int threads, size_t smem, int dev, int* out) {
  static std::unordered_map<const void*, std::unordered_map<int, int>> cache;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) {
      auto jt = it->second.find(dev);
      if (jt != it->second.end()) {
        *out = jt->second;
        return cudaSuccess;
      }
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int n = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (n < 1) return cudaErrorInvalidConfiguration;
  std::lock_guard<std::mutex> lk(g_mu);
  cache[kernel][dev] = n;
  *out = n;
  return cudaSuccess;
}

int nspec_of(const Tables& t) { return t.num_symbols <= 4 ? 4 : (t.num_symbols <= 8 ? 8 : 16); }

bool column_ok(const pp_column& c, uint32_t type) {
  if (type == PP_SKIP) return true;  // nothing is stored for it
  if (c.validity == nullptr || c.values == nullptr) return false;
  if (type == PP_STRING) return c.offsets != nullptr;
  return true;
}

// Scratch of one job, carved from one stream-ordered allocation.
struct ScratchPlan {
  size_t st_state, st_rc, st_bytes, fail, null_, misc, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

ScratchPlan plan_scratch(size_t base, uint64_t ntiles, uint32_t ns, uint32_t nn, uint64_t bit_words) {
  ScratchPlan p;
  size_t o = align_up(base, 256);
  p.misc = o; o = align_up(o + sizeof(Misc), 256);
  p.st_state = o; o = align_up(o + 8 * ntiles, 256);
  p.st_rc = o; o = align_up(o + 8 * ntiles, 256);
  p.st_bytes = o; o = align_up(o + 8 * ntiles * ns, 256);
  p.fail = o; o = align_up(o + 4 * bit_words, 256);
  p.null_ = o; o = align_up(o + 4 * bit_words * nn, 256);
  p.total = o;
  return p;
}

void fill_job(Job& J, const ScratchPlan& p, uint8_t* scratch) {
  J.misc = reinterpret_cast<Misc*>(scratch + p.misc);
  J.st_state = reinterpret_cast<uint64_t*>(scratch + p.st_state);
  J.st_rc = reinterpret_cast<uint64_t*>(scratch + p.st_rc);
  J.st_bytes = reinterpret_cast<uint64_t*>(scratch + p.st_bytes);
  J.fail_bits = reinterpret_cast<uint32_t*>(scratch + p.fail);
  J.null_bits = reinterpret_cast<uint32_t*>(scratch + p.null_);
}

pp_status check_columns(const pp_parser* P, const pp_columns* out) {
  if (out == nullptr || out->result == nullptr || out->row_valid == nullptr) return PP_E_ARG;
  if (out->num_columns != P->tab.num_columns) return PP_E_ARG;
  for (uint32_t c = 0; c < out->num_columns; ++c)
    if (!column_ok(out->cols[c], P->types[c])) return PP_E_ARG;
  return PP_OK;
}

pp_status map_err(cudaError_t e) {
  if (e == cudaSuccess) return PP_OK;
  if (e == cudaErrorMemoryAllocation) return PP_E_NOMEM;
  return PP_E_CUDA;
}

#ifdef PP_PHASE_TIMING
unsigned long long* g_phase_cycles = nullptr;  // profiling builds: per-phase cycle totals
int g_last_grid = 0, g_last_per_sm = 0;
#endif

// Launches init, tile and finalize kernels for a prepared launch.
// units: some job reads UTF-16LE code units (the kernel form that can).
pp_status run_launch(Launch& L, const ShapeInfo& shape, int nspec, int64_t grid_limit,
                     const pp_parser* timing, cudaStream_t stream, uint32_t max_jobs_y,
                     uint64_t max_tiles, uint64_t max_words, bool units) {
  if (units && shape.units_kernel == nullptr) return PP_E_UNSUPPORTED;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return map_err(e);
  DeviceProps props;
  if ((e = device_props(dev, &props)) != cudaSuccess) return map_err(e);

  const uint32_t gy = std::max<uint32_t>(1, std::min<uint32_t>(max_jobs_y, 65535));
  const uint32_t gx_init = static_cast<uint32_t>(
      std::max<uint64_t>(1, std::min<uint64_t>((std::max(max_tiles, max_words) + kBlockInit - 1) / kBlockInit, 1024)));
  pp_init_kernel<<<dim3(gx_init, gy), kBlockInit, 0, stream>>>(L);
  if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);

#ifdef PP_PHASE_TIMING
  if (g_phase_cycles == nullptr) {
    cudaMalloc(reinterpret_cast<void**>(&g_phase_cycles), 32 * sizeof(unsigned long long));
    cudaMemset(g_phase_cycles, 0, 32 * sizeof(unsigned long long));
  }
  L.phase_cycles = g_phase_cycles;
#endif
  if (L.total_tiles > 0) {
    const void* kern = units ? shape.units_kernel(nspec) : shape.kernel(nspec);
    int per_sm = 0;
    if ((e = kernel_occupancy(kern, shape.threads, shape.smem_bytes, dev, &per_sm)) != cudaSuccess)
      return map_err(e);
    uint64_t grid = std::min<uint64_t>(L.total_tiles, static_cast<uint64_t>(per_sm) * props.sms);
    if (grid_limit > 0) grid = std::min<uint64_t>(grid, static_cast<uint64_t>(grid_limit));
#ifdef PP_PHASE_TIMING
    g_last_grid = static_cast<int>(grid);
    g_last_per_sm = per_sm;
#endif
    if (timing && timing->ev_start) cudaEventRecord(timing->ev_start, stream);
    void* args[] = {&L};
    e = cudaLaunchKernel(kern, dim3(static_cast<uint32_t>(grid)), dim3(shape.threads), args,
                         shape.smem_bytes, stream);
    if (e != cudaSuccess) return map_err(e);
    if (timing && timing->ev_stop) cudaEventRecord(timing->ev_stop, stream);
  }

  const uint32_t gx_fin = static_cast<uint32_t>(
      std::max<uint64_t>(1, std::min<uint64_t>((max_words + kBlockFinal - 1) / kBlockFinal, 1024)));
  pp_finalize_kernel<<<dim3(gx_fin, gy), kBlockFinal, 0, stream>>>(L);
  if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);
  return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

// ============================================================== the ABI ===

#ifdef PP_PHASE_TIMING
// Profiling builds only (not part of include/parparaw.h): copies the
// accumulated per-phase cycle totals of the tile kernel to out[0..31].
extern "C" int parparaw_debug_phase_cycles(unsigned long long* out, int reset) {
  if (g_phase_cycles == nullptr) return -1;
  cudaDeviceSynchronize();
  cudaMemcpy(out, g_phase_cycles, 32 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (reset) cudaMemset(g_phase_cycles, 0, 32 * sizeof(unsigned long long));
  return 0;
}
extern "C" int parparaw_debug_last_launch(int* grid, int* per_sm) {
  *grid = g_last_grid;
  *per_sm = g_last_per_sm;
  return 0;
}
#endif

extern "C" const char* parparaw_status_string(int status) {
  switch (status) {
    case PP_OK: return "ok";
    case PP_E_ARG: return "invalid argument";
    case PP_E_NOMEM: return "out of memory";
    case PP_E_CUDA: return "CUDA error";
    case PP_E_INVALID_INPUT: return "input entered the invalid state";
    case PP_E_UNTERMINATED: return "input ended in a non-accepting state";
    case PP_E_CAPACITY: return "output capacity exceeded";
    case PP_E_TIMEOUT: return "device wait timed out";
    case PP_E_BAD_TABLE: return "malformed DFA, symbol groups or schema";
    case PP_E_UNSUPPORTED: return "limit of this build exceeded";
    default: return "unknown status";
  }
}

extern "C" pp_status parparaw_create(const pp_dfa* dfa, const pp_symbol_groups* groups,
                                     const pp_schema* schema, pp_parser** out) {
  if (out == nullptr) return PP_E_ARG;
  *out = nullptr;
  if (dfa == nullptr || groups == nullptr || schema == nullptr) return PP_E_ARG;
  if (dfa->transitions == nullptr || dfa->emit == nullptr) return PP_E_ARG;
  const uint32_t S = dfa->num_states, G = dfa->num_groups;
  if (S == 0 || G == 0) return PP_E_BAD_TABLE;
  if (S > PP_MAX_STATES || G > PP_MAX_GROUPS) return PP_E_UNSUPPORTED;
  if (dfa->start_state >= S) return PP_E_BAD_TABLE;
  if (dfa->invalid_state != PP_NO_STATE && dfa->invalid_state >= S) return PP_E_BAD_TABLE;
  if (groups->catch_all >= G) return PP_E_BAD_TABLE;
  if (groups->num_symbols > PP_MAX_SYMBOLS) return PP_E_UNSUPPORTED;
  if (groups->num_symbols > 0 && (groups->symbols == nullptr || groups->groups == nullptr)) return PP_E_ARG;
  if (schema->num_columns == 0 || schema->types == nullptr) return PP_E_BAD_TABLE;
  if (schema->num_columns > PP_MAX_COLUMNS) return PP_E_UNSUPPORTED;

  pp_parser* P = new (std::nothrow) pp_parser();
  if (P == nullptr) return PP_E_NOMEM;
  Tables& T = P->tab;
  std::memset(&T, 0, sizeof(T));
  for (uint32_t g = 0; g < G; ++g) {
    uint64_t row = 0;
    uint32_t em = 0;
    for (uint32_t s = 0; s < PP_MAX_STATES; ++s) {
      uint32_t nxt = s, tag = PP_TAG_CONTROL;
      if (s < S) {
        nxt = dfa->transitions[g * S + s];
        tag = dfa->emit[g * S + s];
        if (nxt >= S || tag > PP_TAG_CONTROL) { delete P; return PP_E_BAD_TABLE; }
      }
      row |= static_cast<uint64_t>(nxt) << (8 * s);
      em |= tag << (2 * s);
    }
    T.trans[g] = row;
    T.emit[g] = em;
  }
  if (dfa->invalid_state != PP_NO_STATE) {
    const uint32_t inv = dfa->invalid_state;
    for (uint32_t g = 0; g < G; ++g) {
      if (((T.trans[g] >> (8 * inv)) & 0xFF) != inv || ((T.emit[g] >> (2 * inv)) & 3u) != PP_TAG_CONTROL) {
        delete P;
        return PP_E_BAD_TABLE;  // the invalid state must absorb and emit nothing
      }
    }
  }
  bool seen[256] = {false};
  for (int b = 0; b < 256; ++b) T.group_of[b] = groups->catch_all;
  for (uint32_t i = 0; i < groups->num_symbols; ++i) {
    const uint8_t b = groups->symbols[i], g = groups->groups[i];
    if (seen[b] || g >= G || g == groups->catch_all) { delete P; return PP_E_BAD_TABLE; }
    seen[b] = true;
    T.group_of[b] = g;
    T.rep[i] = 0x01010101u * b;
  }
  // composite of a catch-all run followed by each group: (T_* o T_g)_i = T_g[T_*[i]]
  const uint64_t tca = T.trans[groups->catch_all];
  for (uint32_t g = 0; g < PP_MAX_GROUPS; ++g) {
    uint64_t row = 0;
    for (uint32_t s = 0; s < PP_MAX_STATES; ++s) {
      const uint32_t mid = (tca >> (8 * s)) & 0xFF;
      row |= ((T.trans[g] >> (8 * mid)) & 0xFFull) << (8 * s);
    }
    T.trans_run[g] = row;
  }
  // one-lookup steps of the re-simulation (see Tables::step)
  for (uint32_t r = 0; r < 2; ++r)
    for (uint32_t g = 0; g < PP_MAX_GROUPS; ++g)
      for (uint32_t s0 = 0; s0 < PP_MAX_STATES; ++s0) {
        const uint32_t inv = dfa->invalid_state;
        uint32_t s1 = s0;
        bool slow = false;
        if (r) {
          s1 = (tca >> (8 * s0)) & 0xFF;
          const uint32_t e_ca = T.emit[groups->catch_all];
          const uint32_t tag0 = (e_ca >> (2 * s0)) & 3u, tagr = (e_ca >> (2 * s1)) & 3u;
          slow = tag0 != PP_TAG_DATA || tagr != PP_TAG_DATA || (s0 != inv && s1 == inv);
        }
        const uint32_t ns = (T.trans[g] >> (8 * s1)) & 0xFF;
        const uint32_t tag = (T.emit[g] >> (2 * s1)) & 3u;
        const bool enters_inv = s1 != inv && ns == inv;
        T.step[r][g][s0] = static_cast<uint8_t>(ns | (tag << 3) | (enters_inv ? kStepInv : 0) | (slow ? kStepSlow : 0));
      }
  bool idem = true;
  for (uint32_t s = 0; s < S; ++s) {
    const uint32_t once = (tca >> (8 * s)) & 0xFF;
    if (((tca >> (8 * once)) & 0xFF) != once) idem = false;
  }
  T.idempotent = idem ? 1 : 0;
  T.num_states = static_cast<uint8_t>(S);
  T.num_groups = static_cast<uint8_t>(G);
  T.num_symbols = static_cast<uint8_t>(groups->num_symbols);
  T.catch_all = groups->catch_all;
  T.start_state = dfa->start_state;
  T.invalid_state = dfa->invalid_state;
  T.accept_mask = dfa->accept_mask;
  T.num_columns = static_cast<uint8_t>(schema->num_columns);
  uint32_t ns = 0, nn = 0;
  for (uint32_t c = 0; c < schema->num_columns; ++c) {
    const uint32_t ty = schema->types[c];
    if (ty > PP_SKIP) { delete P; return PP_E_BAD_TABLE; }
    P->types[c] = ty;
    T.col_type[c] = static_cast<uint8_t>(ty);
    T.str_slot[c] = 0xFF;
    T.num_slot[c] = 0xFF;
    if (ty == PP_STRING) {
      if (ns >= PP_MAX_STRING_COLUMNS) { delete P; return PP_E_UNSUPPORTED; }
      T.str_slot[c] = static_cast<uint8_t>(ns++);
    } else if (ty != PP_SKIP) {
      T.num_slot[c] = static_cast<uint8_t>(nn++);
    }
  }
  T.num_str = static_cast<uint8_t>(ns);
  T.num_num = static_cast<uint8_t>(nn);
  *out = P;
  return PP_OK;
}

extern "C" void parparaw_destroy(pp_parser* parser) { delete parser; }

extern "C" pp_status parparaw_set_option(pp_parser* P, pp_option option, int64_t value) {
  if (P == nullptr) return PP_E_ARG;
  switch (option) {
    case PP_OPT_TILE_CONFIG:
      if (value < 0 || value > 14) return PP_E_ARG;
      P->tile_config = static_cast<int>(value);
      return PP_OK;
    case PP_OPT_TIMEOUT_MS:
      if (value <= 0) return PP_E_ARG;
      P->timeout_ns = static_cast<uint64_t>(value) * 1000000ull;
      return PP_OK;
    case PP_OPT_GRID_LIMIT:
      if (value < 0) return PP_E_ARG;
      P->grid_limit = value;
      return PP_OK;
    case PP_OPT_PARTIAL_INPUT:
      if (value != 0 && value != 1) return PP_E_ARG;
      P->tab.partial = static_cast<uint8_t>(value);
      return PP_OK;
    case PP_OPT_FIRST_ITEM:
      if (value < 0 || value > 0xFFFFFFFFll) return PP_E_ARG;
      P->first_item = static_cast<uint32_t>(value);
      return PP_OK;
    case PP_OPT_SKIP_RECORDS:
      if (value < 0 || value > 0xFFFFFFFFll) return PP_E_ARG;
      P->tab.skip_records = static_cast<uint32_t>(value);
      return PP_OK;
    case PP_OPT_UTF16LE: {
      if (value != 0 && value != 1) return PP_E_ARG;
      if (value == 1) {
        // code units read one at a time parse a surrogate pair as one symbol
        // when the catch-all transition is idempotent and keeps its tag
        const Tables& T = P->tab;
        const uint64_t tca = T.trans[T.catch_all];
        const uint32_t eca = T.emit[T.catch_all];
        if (!T.idempotent) return PP_E_UNSUPPORTED;
        for (uint32_t s0 = 0; s0 < T.num_states; ++s0) {
          const uint32_t s1 = (tca >> (8 * s0)) & 0xFF;
          if (((eca >> (2 * s0)) & 3u) != ((eca >> (2 * s1)) & 3u)) return PP_E_UNSUPPORTED;
        }
      }
      P->tab.unit2 = static_cast<uint8_t>(value);
      return PP_OK;
    }
    default:
      return PP_E_ARG;
  }
}

extern "C" pp_status parparaw_get_info(const pp_parser* P, pp_parser_info* info) {
  if (P == nullptr || info == nullptr) return PP_E_ARG;
  const ShapeInfo sh = shape_for(P->tile_config);
  info->num_states = P->tab.num_states;
  info->num_groups = P->tab.num_groups;
  info->num_symbols = P->tab.num_symbols;
  info->num_columns = P->tab.num_columns;
  info->num_string_columns = P->tab.num_str;
  info->catch_all_idempotent = P->tab.idempotent;
  info->tile_bytes = static_cast<uint32_t>(sh.tile_bytes);
  info->threads_per_block = static_cast<uint32_t>(sh.threads);
  return PP_OK;
}

extern "C" pp_status parparaw_set_kernel_events(pp_parser* P, void* start_event, void* stop_event) {
  if (P == nullptr || ((start_event == nullptr) != (stop_event == nullptr))) return PP_E_ARG;
  P->ev_start = static_cast<cudaEvent_t>(start_event);
  P->ev_stop = static_cast<cudaEvent_t>(stop_event);
  return PP_OK;
}

extern "C" pp_status parparaw_infer(const pp_parser* P, const uint8_t* input, uint64_t len,
                                    pp_inference* result, void* stream_) {
  if (P == nullptr || result == nullptr || (input == nullptr && len > 0)) return PP_E_ARG;
  if (P->tab.unit2) return PP_E_UNSUPPORTED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const ShapeInfo shape = shape_for(0);
  if (shape.infer_kernel == nullptr) return PP_E_UNSUPPORTED;
  Launch* Lp = new (std::nothrow) Launch();
  if (Lp == nullptr) return PP_E_NOMEM;
  Launch& L = *Lp;
  std::memset(&L, 0, sizeof(L));
  // the parser's DFA; PP_MAX_COLUMNS field positions, none of them stored
  L.tables0 = P->tab;
  L.tables0.num_columns = PP_MAX_COLUMNS;
  L.tables0.num_str = 0;
  L.tables0.num_num = 0;
  L.tables0.partial = 0;
  for (int c = 0; c < PP_MAX_COLUMNS; ++c) {
    L.tables0.col_type[c] = PP_STRING;
    L.tables0.str_slot[c] = 0xFF;
    L.tables0.num_slot[c] = 0xFF;
  }
  Job& J = L.job0;
  J.input = input;
  J.len = len;
  J.head = len > 0 ? (reinterpret_cast<uintptr_t>(input) & 15u) : 0;
  J.ntiles = len > 0 ? (J.head + len + shape.tile_bytes - 1) / shape.tile_bytes : 0;
  J.tile_base = 0;
  J.rows_cap = ~0ull;  // no row is stored
  J.bit_words = 0;
  J.row_valid = nullptr;
  J.result = nullptr;
  const ScratchPlan plan = plan_scratch(64, J.ntiles, 0, 0, 0);
  uint8_t* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), plan.total, stream);
  if (e != cudaSuccess) {
    delete Lp;
    return map_err(e);
  }
  fill_job(J, plan, scratch);
  L.njobs = 1;
  L.total_tiles = J.ntiles;
  L.work_counter = reinterpret_cast<unsigned long long*>(scratch);
  L.first_item = 0;
  L.timeout_ns = P->timeout_ns;
  pp_status st = PP_OK;
  int dev = 0;
  DeviceProps props;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || (e = device_props(dev, &props)) != cudaSuccess) {
    st = map_err(e);
  } else {
    const uint32_t gx_init = static_cast<uint32_t>(
        std::max<uint64_t>(1, std::min<uint64_t>((J.ntiles + kBlockInit - 1) / kBlockInit, 1024)));
    pp_init_kernel<<<gx_init, kBlockInit, 0, stream>>>(L);
    e = cudaGetLastError();
    if (e == cudaSuccess && L.total_tiles > 0) {
      const void* kern = shape.infer_kernel(nspec_of(P->tab));
      int per_sm = 0;
      if ((e = kernel_occupancy(kern, shape.threads, shape.smem_bytes, dev, &per_sm)) == cudaSuccess) {
        const uint64_t grid = std::min<uint64_t>(L.total_tiles, static_cast<uint64_t>(per_sm) * props.sms);
        void* args[] = {&L};
        e = cudaLaunchKernel(kern, dim3(static_cast<uint32_t>(grid)), dim3(shape.threads), args,
                             shape.smem_bytes, stream);
      }
    }
    if (e == cudaSuccess) {
      pp_infer_finalize_kernel<<<1, PP_MAX_COLUMNS, 0, stream>>>(L, result);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = map_err(e);
  }
  cudaFreeAsync(scratch, stream);
  delete Lp;
  return st;
}

// UTF-16LE inputs are whole code units at an even address.
static bool units_ok(const pp_parser* P, const uint8_t* input, uint64_t len) {
  return !P->tab.unit2 || ((len % 2) == 0 && (reinterpret_cast<uintptr_t>(input) % 2) == 0);
}

// The scratch (bytes) that one parse of len bytes into rows_cap rows needs.
size_t pp_parse_scratch_bytes(const pp_parser* P, uint64_t len, uint64_t rows_cap) {
  const ShapeInfo shape = shape_for(P->tile_config);
  const uint64_t ntiles = len > 0 ? (15 + len + shape.tile_bytes - 1) / shape.tile_bytes : 0;  // any alignment
  return plan_scratch(64, ntiles, P->tab.num_str, P->tab.num_num, (rows_cap + 31) / 32 + 1).total;
}

// parparaw_parse with the scratch either allocated stream-ordered here
// (scratch == nullptr) or taken from the caller's device block.
pp_status pp_parse_with_scratch(const pp_parser* P, const uint8_t* input, uint64_t len, const pp_columns* out,
                                cudaStream_t stream, uint8_t* scratch_block, size_t scratch_cap) {
  if (P == nullptr || (input == nullptr && len > 0)) return PP_E_ARG;
  if (!units_ok(P, input, len)) return PP_E_ARG;
  pp_status st = check_columns(P, out);
  if (st != PP_OK) return st;
  const ShapeInfo shape = shape_for(P->tile_config);

  Launch* Lp = new (std::nothrow) Launch();
  if (Lp == nullptr) return PP_E_NOMEM;
  Launch& L = *Lp;
  std::memset(&L, 0, sizeof(L));
  Job& J = L.job0;
  J.input = input;
  J.len = len;
  J.head = len > 0 ? (reinterpret_cast<uintptr_t>(input) & 15u) : 0;
  J.ntiles = len > 0 ? (J.head + len + shape.tile_bytes - 1) / shape.tile_bytes : 0;
  J.tile_base = 0;
  J.rows_cap = out->rows_cap;
  J.bit_words = (out->rows_cap + 31) / 32 + 1;
  J.row_valid = out->row_valid;
  J.result = out->result;
  L.tables0 = P->tab;
  for (uint32_t c = 0; c < out->num_columns; ++c) {
    L.cols0[c].values = out->cols[c].values;
    L.cols0[c].offsets = out->cols[c].offsets;
    L.cols0[c].validity = out->cols[c].validity;
    L.cols0[c].values_cap = out->cols[c].values_cap;
  }
  const ScratchPlan plan = plan_scratch(64, J.ntiles, P->tab.num_str, P->tab.num_num, J.bit_words);
  uint8_t* scratch = scratch_block;
  if (scratch_block != nullptr) {
    if (plan.total > scratch_cap) {
      delete Lp;
      return PP_E_UNSUPPORTED;
    }
  } else {
    const cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), plan.total, stream);
    if (e != cudaSuccess) {
      delete Lp;
      return map_err(e);
    }
  }
  fill_job(J, plan, scratch);
  L.jobs = nullptr;
  L.cols = nullptr;
  L.tables = nullptr;
  L.njobs = 1;
  L.total_tiles = J.ntiles;
  L.work_counter = reinterpret_cast<unsigned long long*>(scratch);
  L.first_item = P->first_item;
  L.timeout_ns = P->timeout_ns;
  st = run_launch(L, shape, nspec_of(P->tab), P->grid_limit, P, stream, 1, J.ntiles, J.bit_words,
                  P->tab.unit2 != 0);
  if (scratch_block == nullptr) cudaFreeAsync(scratch, stream);
  delete Lp;
  return st;
}

extern "C" pp_status parparaw_parse(const pp_parser* P, const uint8_t* input, uint64_t len,
                                    const pp_columns* out, void* stream_) {
  return pp_parse_with_scratch(P, input, len, out, static_cast<cudaStream_t>(stream_), nullptr, 0);
}

namespace pp {
namespace {

// Host-side description of a batch: unique parser tables, one job per item,
// the items' columns, and where every piece lives in one device allocation
// laid out as [per-job scratch][tables][jobs][columns].
struct BatchPlan {
  std::vector<Tables> tables;
  std::vector<Job> jobs;
  std::vector<Col> cols;
  std::vector<ScratchPlan> plans;
  const pp_parser* first = nullptr;
  ShapeInfo shape;
  int nspec = 4;
  bool units = false;  // some item reads UTF-16LE code units
  uint64_t total_tiles = 0, max_tiles = 0, max_words = 0;
  size_t off_tables = 0, off_jobs = 0, off_cols = 0, total = 0;
};

pp_status plan_batch(const pp_batch_item* items, uint64_t n, BatchPlan* bp) {
  if (items == nullptr || n == 0) return PP_E_ARG;
  if (n > 0xFFFFFFFFull) return PP_E_UNSUPPORTED;
  bp->first = items[0].parser;
  if (bp->first == nullptr) return PP_E_ARG;
  bp->shape = shape_for(bp->first->tile_config);
  std::unordered_map<const pp_parser*, uint32_t> table_index;
  bp->jobs.resize(n);
  bp->plans.resize(n);
  size_t scratch_bytes = 64;
  for (uint64_t i = 0; i < n; ++i) {
    const pp_batch_item& it = items[i];
    if (it.parser == nullptr || (it.input == nullptr && it.len > 0)) return PP_E_ARG;
    if (!units_ok(it.parser, it.input, it.len)) return PP_E_ARG;
    const pp_status st = check_columns(it.parser, it.out);
    if (st != PP_OK) return st;
    auto found = table_index.find(it.parser);
    uint32_t ti;
    if (found == table_index.end()) {
      ti = static_cast<uint32_t>(bp->tables.size());
      bp->tables.push_back(it.parser->tab);
      table_index[it.parser] = ti;
      bp->nspec = std::max(bp->nspec, nspec_of(it.parser->tab));
      bp->units = bp->units || it.parser->tab.unit2 != 0;
    } else {
      ti = found->second;
    }
    Job& J = bp->jobs[i];
    std::memset(&J, 0, sizeof(J));
    J.input = it.input;
    J.len = it.len;
    J.head = it.len > 0 ? (reinterpret_cast<uintptr_t>(it.input) & 15u) : 0;
    J.ntiles = it.len > 0 ? (J.head + it.len + bp->shape.tile_bytes - 1) / bp->shape.tile_bytes : 0;
    J.tile_base = bp->total_tiles;
    J.rows_cap = it.out->rows_cap;
    J.bit_words = (it.out->rows_cap + 31) / 32 + 1;
    J.row_valid = it.out->row_valid;
    J.result = it.out->result;
    J.tables = ti;
    J.col0 = static_cast<uint32_t>(bp->cols.size());
    for (uint32_t c = 0; c < it.out->num_columns; ++c) {
      Col col;
      col.values = it.out->cols[c].values;
      col.offsets = it.out->cols[c].offsets;
      col.validity = it.out->cols[c].validity;
      col.values_cap = it.out->cols[c].values_cap;
      bp->cols.push_back(col);
    }
    bp->plans[i] = plan_scratch(scratch_bytes, J.ntiles, it.parser->tab.num_str, it.parser->tab.num_num,
                                J.bit_words);
    scratch_bytes = bp->plans[i].total;
    bp->total_tiles += J.ntiles;
    bp->max_tiles = std::max(bp->max_tiles, J.ntiles);
    bp->max_words = std::max(bp->max_words, J.bit_words);
  }
  bp->off_tables = align_up(scratch_bytes, 256);
  bp->off_jobs = align_up(bp->off_tables + sizeof(Tables) * bp->tables.size(), 256);
  bp->off_cols = align_up(bp->off_jobs + sizeof(Job) * bp->jobs.size(), 256);
  bp->total = align_up(bp->off_cols + sizeof(Col) * bp->cols.size(), 256);
  return PP_OK;
}

// Points the jobs at their scratch in `dev` and packs tables, jobs and
// columns into one host image of the device region starting at off_tables.
void pack_batch(BatchPlan& bp, uint8_t* dev, std::vector<uint8_t>* image) {
  for (size_t i = 0; i < bp.jobs.size(); ++i) fill_job(bp.jobs[i], bp.plans[i], dev);
  image->assign(bp.total - bp.off_tables, 0);
  std::memcpy(image->data(), bp.tables.data(), sizeof(Tables) * bp.tables.size());
  std::memcpy(image->data() + (bp.off_jobs - bp.off_tables), bp.jobs.data(), sizeof(Job) * bp.jobs.size());
  std::memcpy(image->data() + (bp.off_cols - bp.off_tables), bp.cols.data(), sizeof(Col) * bp.cols.size());
}

void batch_launch_params(const BatchPlan& bp, uint8_t* dev, Launch* L) {
  std::memset(L, 0, sizeof(*L));
  L->tables = reinterpret_cast<const Tables*>(dev + bp.off_tables);
  L->jobs = reinterpret_cast<const Job*>(dev + bp.off_jobs);
  L->cols = reinterpret_cast<const Col*>(dev + bp.off_cols);
  L->njobs = static_cast<uint32_t>(bp.jobs.size());
  L->total_tiles = bp.total_tiles;
  L->work_counter = reinterpret_cast<unsigned long long*>(dev);
  L->first_item = bp.first->first_item;
  L->timeout_ns = bp.first->timeout_ns;
}

}  // namespace
}  // namespace pp

struct pp_batch {
  pp::BatchPlan plan;
  uint8_t* dev = nullptr;
  pp::Launch* launch = nullptr;
};

extern "C" pp_status parparaw_parse_batch(const pp_batch_item* items, uint64_t n, void* stream_) {
  if (items == nullptr && n > 0) return PP_E_ARG;
  if (n == 0) return PP_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  BatchPlan bp;
  pp_status st = plan_batch(items, n, &bp);
  if (st != PP_OK) return st;
  uint8_t* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bp.total, stream);
  if (e != cudaSuccess) return map_err(e);
  std::vector<uint8_t> image;
  pack_batch(bp, scratch, &image);
  // pageable source: staged by the runtime before the call returns
  e = cudaMemcpyAsync(scratch + bp.off_tables, image.data(), image.size(), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(scratch, stream);
    return map_err(e);
  }
  Launch* Lp = new (std::nothrow) Launch();
  if (Lp == nullptr) {
    cudaFreeAsync(scratch, stream);
    return PP_E_NOMEM;
  }
  batch_launch_params(bp, scratch, Lp);
  st = run_launch(*Lp, bp.shape, bp.nspec, bp.first->grid_limit, bp.first, stream,
                  static_cast<uint32_t>(std::min<uint64_t>(n, 65535)), bp.max_tiles, bp.max_words, bp.units);
  cudaFreeAsync(scratch, stream);
  delete Lp;
  return st;
}

extern "C" pp_status parparaw_batch_create(const pp_batch_item* items, uint64_t n, pp_batch** out) {
  if (out == nullptr) return PP_E_ARG;
  *out = nullptr;
  pp_batch* b = new (std::nothrow) pp_batch();
  if (b == nullptr) return PP_E_NOMEM;
  pp_status st = plan_batch(items, n, &b->plan);
  if (st != PP_OK) {
    delete b;
    return st;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->dev), b->plan.total);
  if (e != cudaSuccess) {
    delete b;
    return map_err(e);
  }
  std::vector<uint8_t> image;
  pack_batch(b->plan, b->dev, &image);
  e = cudaMemcpy(b->dev + b->plan.off_tables, image.data(), image.size(), cudaMemcpyHostToDevice);
  b->launch = new (std::nothrow) Launch();
  if (e != cudaSuccess || b->launch == nullptr) {
    cudaFree(b->dev);
    delete b->launch;
    delete b;
    return e != cudaSuccess ? map_err(e) : PP_E_NOMEM;
  }
  batch_launch_params(b->plan, b->dev, b->launch);
  *out = b;
  return PP_OK;
}

extern "C" pp_status parparaw_batch_launch(pp_batch* b, void* stream_) {
  if (b == nullptr) return PP_E_ARG;
  const BatchPlan& bp = b->plan;
  return run_launch(*b->launch, bp.shape, bp.nspec, bp.first->grid_limit, bp.first,
                    static_cast<cudaStream_t>(stream_),
                    static_cast<uint32_t>(std::min<uint64_t>(bp.jobs.size(), 65535)), bp.max_tiles, bp.max_words,
                    bp.units);
}

extern "C" void parparaw_batch_destroy(pp_batch* b) {
  if (b == nullptr) return;
  cudaFree(b->dev);
  delete b->launch;
  delete b;
}

// ================================================= allocation-free parse ===
//
// parparaw_parse_noalloc: the same init / tile / finalize kernels as
// parparaw_parse, with the scratch taken from a fixed array in device memory
// instead of a stream-ordered allocation.  See include/parparaw.h.

namespace pp {
namespace {

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[PP_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
uint8_t* g_noalloc_dev_ptr[kNoallocMaxDevices] = {};

// The array's name is only a host-side handle; kernels need its device
// address, looked up once per device with that device current.
cudaError_t noalloc_scratch_ptr(int dev, uint8_t** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_dev_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_dev_ptr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_noalloc_dev_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pp

extern "C" pp_status parparaw_parse_noalloc(const pp_parser* P, const uint8_t* input, uint64_t len,
                                            const pp_columns* out, void* stream_) {
  if (P == nullptr || (input == nullptr && len > 0)) return PP_E_ARG;
  if (!units_ok(P, input, len)) return PP_E_ARG;
  pp_status st = check_columns(P, out);
  if (st != PP_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return map_err(e);
  if (dev < 0 || dev >= kNoallocMaxDevices) return PP_E_UNSUPPORTED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const ShapeInfo shape = shape_for(P->tile_config);

  Launch L;  // on the stack: no host allocation either
  std::memset(&L, 0, sizeof(L));
  Job& J = L.job0;
  J.input = input;
  J.len = len;
  J.head = len > 0 ? (reinterpret_cast<uintptr_t>(input) & 15u) : 0;
  J.ntiles = len > 0 ? (J.head + len + shape.tile_bytes - 1) / shape.tile_bytes : 0;
  J.rows_cap = out->rows_cap;
  J.bit_words = (out->rows_cap + 31) / 32 + 1;
  J.row_valid = out->row_valid;
  J.result = out->result;
  const ScratchPlan plan = plan_scratch(64, J.ntiles, P->tab.num_str, P->tab.num_num, J.bit_words);
  if (plan.total > PP_NOALLOC_SCRATCH_BYTES) return PP_E_UNSUPPORTED;  // input or rows_cap too large
  uint8_t* scratch = nullptr;
  if ((e = noalloc_scratch_ptr(dev, &scratch)) != cudaSuccess) return map_err(e);
  L.tables0 = P->tab;
  for (uint32_t c = 0; c < out->num_columns; ++c) {
    L.cols0[c].values = out->cols[c].values;
    L.cols0[c].offsets = out->cols[c].offsets;
    L.cols0[c].validity = out->cols[c].validity;
    L.cols0[c].values_cap = out->cols[c].values_cap;
  }
  fill_job(J, plan, scratch);
  L.njobs = 1;
  L.total_tiles = J.ntiles;
  L.work_counter = reinterpret_cast<unsigned long long*>(scratch);
  L.first_item = P->first_item;
  L.timeout_ns = P->timeout_ns;

  // the same launch sequence as parparaw_parse: the init kernel clears
  // everything the tile kernel needs at zero (status words, bitmaps,
  // counters), since the array keeps the previous call's contents
  return run_launch(L, shape, nspec_of(P->tab), P->grid_limit, P, stream, 1, J.ntiles, J.bit_words,
                    P->tab.unit2 != 0);
}
