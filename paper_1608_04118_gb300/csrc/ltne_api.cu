// ltne_api.cu -- host side of the C ABI declared in include/ltne.h: the
// mapping from the paper's dimensionless groups (Sec. 2, Sec. 4) to lattice
// constants, validation, the device workspace layout, CUDA-graph replay of
// time steps, observables, field access and checkpoints.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>
#include <vector>

#include "ltne.h"
#include "ltne_internal.h"
#include "ltne_handle.h"

using namespace ltne;

namespace {

constexpr int kGraphSteps = 32;  // steps per captured graph (even: keeps A-B parity)
constexpr uint64_t kStateMagic = 0x4C544E4553544154ull;  // "LTNESTAT"

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t storage_bytes(int storage) {
  switch (storage) {
    case LTNE_F64: return 8;
    case LTNE_F32: return 4;
    default: return 2;
  }
}

}  // namespace

namespace {

int fail_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LTNE_OK;
  cudaGetLastError();  // clear a sticky launch error from this thread's state
  return LTNE_ERR_CUDA;
}

bool in_open(double v, double lo, double hi) { return v > lo && v < hi && isfinite(v); }

// Host passes over whole fields (checks, conversions, the Ergun mean) in a
// fixed number of contiguous chunks spread over the host cores: fn(c, lo, hi)
// handles chunk c = [lo, hi).  The chunking does not depend on the core
// count, so per-chunk partial results combine identically on any host.
constexpr int kHostChunks = 64;

// Worker threads kept for the life of the process (one per host core but
// the caller's), started at the first large pass: a pass hands out its
// chunks through an atomic counter to the workers and the calling thread
// and returns when all are done.  Thread creation per pass cost about as
// much as the conversions of a staged block.  A pass that finds the pool
// busy (another thread's pass), or runs in a process forked after the
// pool started, runs on the calling thread alone.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  // fn(c) for every c in [0, n); false if the pool could not take the pass
  bool run(int n, const std::function<void(int)>& fn) {
    if (getpid() != pid_ || workers_.empty()) return false;
    std::unique_lock<std::mutex> busy(run_m_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &fn;
      n_ = n;
      next_.store(0);
      active_ = (int)workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    for (int c; (c = next_.fetch_add(1)) < n;) fn(c);
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return active_ == 0; });
    job_ = nullptr;
    return true;
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_)
      if (t.joinable()) t.join();
  }

 private:
  HostPool() : pid_(getpid()) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::min<unsigned>(hw ? hw : 1, kHostChunks);
    for (int t = 1; t < nt; ++t) workers_.emplace_back([this] { work(); });
  }
  void work() {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(int)>* job;
      int n;
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        job = job_;
        n = n_;
      }
      for (int c; (c = next_.fetch_add(1)) < n;) (*job)(c);
      std::lock_guard<std::mutex> lk(m_);
      if (--active_ == 0) done_.notify_one();
    }
  }
  const pid_t pid_;
  std::vector<std::thread> workers_;
  std::mutex run_m_, m_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* job_ = nullptr;
  std::atomic<int> next_{0};
  int n_ = 0, active_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// (min_pool: the smallest n worth waking the pool for)
template <typename F>
void host_chunks(int64_t n, F fn, int64_t min_pool = (int64_t)1 << 18) {
  const int64_t len = (n + kHostChunks - 1) / kHostChunks;
  auto chunk = [&](int c) {
    const int64_t lo = (int64_t)c * len, hi = std::min(n, lo + len);
    if (lo < hi) fn(c, lo, hi);
  };
  if (n >= min_pool && HostPool::get().run(kHostChunks, chunk)) return;
  for (int c = 0; c < kHostChunks; ++c) chunk(c);
}

// Pinned staging of whole fields between host arrays and the device planes:
// rows go in blocks through two pinned buffers, so that converting one block
// on the host overlaps the copy of the other.
constexpr size_t kPinBytes = (size_t)32 << 20;

void release_pinned(ltne_handle* h) {
  for (int k = 0; k < 2; ++k) {
    if (h->pin[k]) cudaFreeHost(h->pin[k]);
    if (h->pin_ev[k]) cudaEventDestroy(h->pin_ev[k]);
    h->pin[k] = nullptr;
    h->pin_ev[k] = nullptr;
  }
  h->pin_bytes = 0;
}

cudaError_t ensure_pinned(ltne_handle* h, size_t row_bytes) {
  const size_t bytes = std::max(row_bytes, kPinBytes);
  if (h->pin_bytes >= bytes) return cudaSuccess;
  release_pinned(h);
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h->pin[k]), bytes,
                                  cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->pin_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      release_pinned(h);
      return e;
    }
  }
  h->pin_bytes = bytes;
  return cudaSuccess;
}

// Host -> device: fill(buf, y0, y1) writes rows [y0, y1) of the field,
// packed (nx values of ec bytes per row), into a pinned buffer and returns
// false on a value it rejects; each block is then copied into the device
// plane at dev (row pitch h->pitch).  Asynchronous on the handle's stream.
template <typename Fill>
int upload_field(ltne_handle* h, char* dev, Fill fill) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t row = (size_t)nx * h->ec, dpitch = (size_t)h->pitch * h->ec;
  cudaError_t e = ensure_pinned(h, row);
  if (e != cudaSuccess) return fail_cuda(e);
  const int rows = (int)std::max<size_t>(1, h->pin_bytes / row);
  int slot = 0;
  for (int y0 = 0; y0 < ny; y0 += rows, slot ^= 1) {
    const int y1 = std::min(ny, y0 + rows);
    e = cudaEventSynchronize(h->pin_ev[slot]);  // its previous copy is done
    if (e != cudaSuccess) return fail_cuda(e);
    if (!fill(h->pin[slot], y0, y1)) {
      cudaStreamSynchronize(h->stream);
      return LTNE_ERR_INVALID_ARG;
    }
    e = cudaMemcpy2DAsync(dev + (size_t)y0 * dpitch, dpitch, h->pin[slot], row, row,
                          (size_t)(y1 - y0), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->pin_ev[slot], h->stream);
    if (e != cudaSuccess) return fail_cuda(e);
  }
  return LTNE_OK;
}

// Device -> host: blocks of rows of the plane at dev are copied into the
// pinned buffers in turn, and drain(buf, y0, y1) converts each block while
// the next one is in flight.  Returns when the whole field is drained.
template <typename Drain>
int download_field(ltne_handle* h, const char* dev, Drain drain) {
  const int nx = h->p.nx, ny = h->p.ny;
  const size_t row = (size_t)nx * h->ec, dpitch = (size_t)h->pitch * h->ec;
  cudaError_t e = ensure_pinned(h, row);
  if (e != cudaSuccess) return fail_cuda(e);
  const int rows = (int)std::max<size_t>(1, h->pin_bytes / row);
  const int nb = (ny + rows - 1) / rows;
  for (int b = 0; b <= nb; ++b) {
    if (b < nb) {
      const int y0 = b * rows, y1 = std::min(ny, y0 + rows);
      e = cudaMemcpy2DAsync(h->pin[b & 1], row, dev + (size_t)y0 * dpitch, dpitch, row,
                            (size_t)(y1 - y0), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(h->pin_ev[b & 1], h->stream);
      if (e != cudaSuccess) return fail_cuda(e);
    }
    if (b > 0) {
      const int y0 = (b - 1) * rows, y1 = std::min(ny, y0 + rows);
      e = cudaEventSynchronize(h->pin_ev[(b - 1) & 1]);
      if (e != cudaSuccess) return fail_cuda(e);
      drain(h->pin[(b - 1) & 1], y0, y1);
    }
  }
  return LTNE_OK;
}

}  // namespace

namespace ltne {

double ergun_mean_of_chunks(const double* part, int64_t n) {
  double acc = 0.0;
  for (int64_t c = 0, m = ergun_chunks(n); c < m; ++c) acc += part[c];
  return acc / (double)n;
}

double ergun_mean(const double* porosity, int64_t n) {
  std::vector<double> part((size_t)ergun_chunks(n));
  host_chunks(
      (int64_t)part.size(),
      [&](int, int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c) {
          double v[kErgunLanes];
          for (int l = 0; l < kErgunLanes; ++l) {
            double s = 0.0;
            for (int j = 0; j < kErgunPerLane; ++j) {
              const int64_t i = c * kErgunChunk + (int64_t)j * kErgunLanes + l;
              if (i < n) s += ergun_term(porosity[i]);
            }
            v[l] = s;
          }
          for (int st = kErgunLanes / 2; st >= 1; st >>= 1)
            for (int l = 0; l < st; ++l) v[l] += v[l + st];
          part[(size_t)c] = v[0];
        }
      },
      64);
  return ergun_mean_of_chunks(part.data(), n);
}

// Lattice constants from the problem statement.  Returns a status code.
int derive_params(const ltne_params& p, const double* erg_mean, NodeParams<double>& P,
                  DerivedInfo& info) {
  const double L = p.ny - 1.0;
  const double cs2 = 1.0 / 3.0;            // c_s^2 (below Eq. 23)
  const double csT2 = p.varpi / 2.0;       // c_sT^2 (below Eq. 49)
  const double uc = p.Ma * sqrt(cs2);      // velocity scale u_c = Ma c_s
  const double dT = p.T_hot - p.T_cold;
  const double gbeta = (p.Ra > 0 && dT != 0) ? uc * uc / (dT * L) : 0.0;  // u_c^2 = g b dT L
  double nu_f;
  if (p.nu_override > 0) nu_f = p.nu_override;
  else if (p.Ra > 0) nu_f = uc * L * sqrt(p.Pr / p.Ra);  // from Ra = g b dT L^3 / (nu a)
  else return LTNE_ERR_INVALID_ARG;
  const double alpha_f = nu_f / p.Pr;
  const double nu_e = p.J_e * nu_f;
  const double alpha_s = p.gamma_sf / p.sigma * alpha_f;
  info.L = L;
  info.nu_f = nu_f;
  info.alpha_f = alpha_f;

  P.rho0 = 1.0;
  P.T0 = p.T_ref;
  P.s_e = p.s_e;
  P.s_eps = p.s_eps;
  P.s_q = p.s_q;
  P.s_nu = 1.0 / (nu_e / cs2 + 0.5);           // Eq. 23
  P.zeta_a = 1.0 / (alpha_f / csT2 + 0.5);     // Eq. 49
  P.zeta_e = p.zeta_e;
  P.zeta_nu = p.zeta_nu;
  P.eta_a = 1.0 / (alpha_s / csT2 + 0.5);      // Eq. 49
  P.eta_e = p.eta_e;
  P.eta_nu = p.eta_nu;
  P.c3 = -4.0 + 5.0 * p.varpi;
  P.wt0 = 1.0 - p.varpi;
  P.wt1 = p.varpi / 4.0;
  P.gbeta = gbeta;
  P.ext_ax = p.ext_ax;
  P.ext_ay = p.ext_ay;
  P.phi_u = p.porosity;
  P.hcoef = p.H * alpha_f / (L * L);           // h_v/(rho c)_f from H_v = h_v L^2/k_f
  P.sigma = p.sigma;
  P.qf = p.qf;
  P.qs = p.qs;
  P.dT_hot = p.T_hot - p.T_ref;
  P.dT_cold = p.T_cold - p.T_ref;
  P.kmode = p.permeability == LTNE_K_ERGUN ? 1 : 0;
  P.fmode = p.F_phi < 0 ? 1 : 0;
  P.Fconst = p.F_phi < 0 ? 0.0 : p.F_phi;
  if (P.kmode == 0) {
    const double K = p.Da * L * L;             // Da = K / L^2
    P.nu_over_K = nu_f / K;
    P.inv_sqrtK = 1.0 / sqrt(K);
    P.erg_a = P.erg_b = P.erg_c = 0.0;
  } else {
    double d = p.d_p;
    if (d <= 0) {
      // mean over the nodes of phi^3 / (1-phi)^2, so that mean K/L^2 = Da
      double acc = 0.0;
      if (erg_mean) {
        acc = *erg_mean;
      } else {
        const double ph = p.porosity;
        acc = ph * ph * ph / ((1 - ph) * (1 - ph));
      }
      d = L * sqrt(150.0 * p.Da / acc);
    }
    info.d_ergun = d;
    P.erg_a = 150.0 * nu_f / (d * d);
    P.erg_b = 1.75 / d;
    P.erg_c = P.Fconst * sqrt(150.0) / d;
    P.nu_over_K = P.inv_sqrtK = 0.0;
  }
  // Coefficients at the uniform porosity (used when no per-node field is
  // set); the same definitions as the device's per-node evaluation.
  {
    Medium<double>& m = P.um;
    const double ph = p.porosity;
    m.phi = ph;
    m.inv_phi = 1.0 / ph;
    m.a = P.hcoef / ph;                                  // Eq. 42
    m.b = P.hcoef / ((1.0 - ph) * p.sigma);
    m.inv_1d = 1.0 / (1.0 + 0.5 * m.a + 0.5 * m.b);      // Eqs. 43-46
    if (P.kmode == 0) {
      m.c0 = P.nu_over_K;
      m.c1 = (P.fmode == 0 ? P.Fconst : 1.75 / sqrt(150.0 * ph * ph * ph)) * P.inv_sqrtK;
    } else {
      const double om = 1.0 - ph, ip3 = 1.0 / (ph * ph * ph);
      m.c0 = P.erg_a * om * om * ip3;
      m.c1 = P.fmode == 1 ? P.erg_b * om * ip3 : P.erg_c * om / (ph * sqrt(ph));
    }
    m.l0 = 0.5 * (1.0 + 0.5 * ph * m.c0);                // Eq. 22
    m.l1 = 0.5 * ph * m.c1;
    m.inv_oms = 1.0 / ((1.0 - ph) * p.sigma);
  }
  // Local h_v (Eq. 52): h_v/(rho c)_f = H_p alpha_f / D_p^2 with
  // H_p = 0.376 (u_m D_p / nu_f)^0.644 Pr^0.37.
  P.hv_local = p.hv_local ? 1 : 0;
  P.tcorr = p.thermal_correction ? 1 : 0;
  {
    const double Dp = p.Dp_over_L * L;
    P.hv_c = p.hv_local ? 0.376 * pow(p.Pr, 0.37) * pow(Dp / nu_f, 0.644) * alpha_f / (Dp * Dp)
                        : 0.0;
  }
  const double rates[] = {P.s_e, P.s_eps, P.s_q, P.s_nu, P.zeta_a, P.zeta_e,
                          P.zeta_nu, P.eta_a, P.eta_e, P.eta_nu};
  for (double r : rates)
    if (!in_open(r, 0.0, 2.0)) return LTNE_ERR_UNSTABLE_TAU;
  return LTNE_OK;
}

int validate_params(const ltne_params& p) {
  if (p.nx < 4 || p.ny < 4) return LTNE_ERR_INVALID_ARG;
  // 19 padded planes must stay below 2^32 elements (32-bit element indices
  // in the kernels): at most about 2.2e8 nodes, e.g. 14800 x 14800.
  {
    const int64_t pitch = ((int64_t)p.nx + 63) / 64 * 64;
    const int64_t plane = (pitch * p.ny + 127) / 128 * 128;
    if (19 * plane >= ((int64_t)1 << 32)) return LTNE_ERR_INVALID_ARG;
  }
  if (p.storage < LTNE_F64 || p.storage > LTNE_BF16DEV) return LTNE_ERR_INVALID_ARG;
  if (p.bc < LTNE_BC_CAVITY || p.bc > LTNE_BC_CHANNEL) return LTNE_ERR_INVALID_ARG;
  if (p.permeability != LTNE_K_DARCY && p.permeability != LTNE_K_ERGUN) return LTNE_ERR_INVALID_ARG;
  if (!in_open(p.porosity, 0.0, 1.0)) return LTNE_ERR_INVALID_ARG;
  if (!in_open(p.varpi, 0.0, 1.0)) return LTNE_ERR_INVALID_ARG;
  if (!(p.Pr > 0) || !(p.sigma > 0) || !(p.J_e > 0) || !(p.gamma_sf > 0)) return LTNE_ERR_INVALID_ARG;
  if (!(p.Da > 0) || !(p.Ma > 0) || !(p.H >= 0) || !(p.Ra >= 0)) return LTNE_ERR_INVALID_ARG;
  if (p.hv_local != 0 && p.hv_local != 1) return LTNE_ERR_INVALID_ARG;
  if (p.thermal_correction != 0 && p.thermal_correction != 1) return LTNE_ERR_INVALID_ARG;
  if (p.hv_local && !(p.Dp_over_L > 0 && isfinite(p.Dp_over_L))) return LTNE_ERR_INVALID_ARG;
  const double vals[] = {p.Ra, p.Pr, p.Da, p.H, p.gamma_sf, p.sigma, p.J_e, p.T_hot, p.T_cold,
                         p.T_ref, p.Ma, p.F_phi, p.d_p, p.qf, p.qs, p.ext_ax, p.ext_ay,
                         p.nu_override};
  for (double v : vals)
    if (!isfinite(v)) return LTNE_ERR_INVALID_ARG;
  return LTNE_OK;
}

// Observables from the reduction accumulators of one lattice.
int finish_observables(const ltne_params& p, const DerivedInfo& info, int64_t step,
                       bool have_prev, const double* acc, ltne_obs* out) {
  const double L = info.L, dT = p.T_hot - p.T_cold, nn = (double)p.nx * p.ny;
  const bool cav = p.bc == LTNE_BC_CAVITY;
  // The planes hold deviations from rho0 = 1 and T0 = T_ref; the reference
  // parts of each sum are added here in FP64.  Over the trapezoid weights
  // (sum L) the wall stencils carry -1.5 T0 L (hot) and +1.5 T0 L (cold).
  const double T0 = p.T_ref;
  out->Nu_f_hot = cav ? (1.5 * (p.T_hot - T0) * L + acc[A_NUF_H]) / dT : 0.0;
  out->Nu_s_hot = cav ? (1.5 * (p.T_hot - T0) * L + acc[A_NUS_H]) / dT : 0.0;
  out->Nu_f_cold = cav ? (-1.5 * (p.T_cold - T0) * L + acc[A_NUF_C]) / dT : 0.0;
  out->Nu_s_cold = cav ? (-1.5 * (p.T_cold - T0) * L + acc[A_NUS_C]) / dT : 0.0;
  auto rel = [](double d2, double x2) { return d2 == 0 ? 0.0 : sqrt(d2 / x2); };
  // |T|^2 = sum (T0 + dT)^2
  const double tf2 = nn * T0 * T0 + 2 * T0 * acc[A_SUMTF] + acc[A_TF2];
  const double ts2 = nn * T0 * T0 + 2 * T0 * acc[A_SUMTS] + acc[A_TS2];
  out->residual = have_prev ? fmax(rel(acc[A_DU2], acc[A_U2]),
                                   fmax(rel(acc[A_DTF2], tf2), rel(acc[A_DTS2], ts2)))
                            : NAN;
  const double sphi = acc[A_SUMPHI];
  out->mass = nn + acc[A_MASS];
  // sum[phi T_f + (1-phi) sigma T_s] - sum[phi Q_f + (1-phi) sigma Q_s]/2
  out->energy = acc[A_ENERGY] + T0 * (sphi + p.sigma * (nn - sphi))
                - 0.5 * (p.qf * sphi + p.sigma * p.qs * (nn - sphi));
  out->max_u = sqrt(acc[A_MAXU]);  // the pass accumulates max |u|^2
  out->max_dT = acc[A_MAXDT];
  out->mean_Tf = T0 + acc[A_SUMTF] / nn;
  out->mean_Ts = T0 + acc[A_SUMTS] / nn;
  out->Fo = info.alpha_f * (double)step / (L * L);
  out->step = step;
  out->nonfinite = (int64_t)acc[A_BAD];
  return out->nonfinite > 0 ? LTNE_ERR_NONFINITE : LTNE_OK;
}

}  // namespace ltne

namespace {

int derive(ltne_handle* h, const double* erg_mean) {
  DerivedInfo info;
  ltne_params pg = h->p;
  if (h->slab) pg.ny = h->gny;  // a slab takes the lattice constants of the whole cavity
  const int rc = derive_params(pg, h->slab ? nullptr : erg_mean, h->P, info);
  if (rc == LTNE_OK) {
    h->L = info.L;
    h->nu_f = info.nu_f;
    h->alpha_f = info.alpha_f;
    h->d_ergun = info.d_ergun;
  }
  return rc;
}

void layout(ltne_handle* h) {
  const ltne_params& p = h->p;
  h->es = storage_bytes(p.storage);
  h->ec = p.storage == LTNE_F64 ? 8 : 4;
  h->pitch = (int64_t)align_up((size_t)p.nx, 64);
  h->plane = (int64_t)align_up((size_t)(h->pitch * p.ny), 128);
  const size_t A = 256;
  size_t off = 0;
  for (int b = 0; b < 2; ++b) {
    h->off_pop[b] = off;
    off = align_up(off + 19 * (size_t)h->plane * h->es, A);
  }
  h->off_phi = off;
  if (p.porosity_field) off = align_up(off + (size_t)h->plane * h->ec, A);
  for (int b = 0; b < 2; ++b) {  // the current fields and the residual snapshot
    h->off_mac[b] = off;
    off = align_up(off + 5 * (size_t)h->plane * h->ec, A);
  }
  h->red_blocks = reduce_blocks(p.nx, p.ny);
  h->off_part = off;
  off = align_up(off + (size_t)h->red_blocks * NACC * sizeof(double), A);
  h->off_out = off;
  off = align_up(off + NACC * sizeof(double), A);
  // two uint32 step counters for the stochastic rounding, the device error
  // word, and the flag set_fields' host-reading kernels raise on a bad value
  h->off_tick = off;
  off = align_up(off + 4 * sizeof(uint32_t), A);
  for (int b = 0; b < 2; ++b) {  // |u| of the previous state per buffer (Eq. 52)
    h->off_um[b] = off;
    if (p.hv_local) off = align_up(off + (size_t)h->plane * h->ec, A);
  }
  for (int k = 0; k < 4; ++k) {  // a slab's halo messages: 5 x nx values each
    h->off_halo[k] = off;
    if (h->slab) off = align_up(off + 5 * (size_t)p.nx * h->es, A);
  }
  h->ws_bytes = off;
  h->enc_scale = p.storage == LTNE_F16DEV ? 1024.0f : 1.0f;  // FP16 deviations x 2^10
}

LatticeArgs lattice_args(const ltne_handle* h, int src_buf, int write_macros) {
  LatticeArgs a{};
  a.src = h->ws + h->off_pop[src_buf];
  a.dst = h->ws + h->off_pop[src_buf ^ 1];
  a.phi = h->p.porosity_field ? h->ws + h->off_phi : nullptr;
  a.mac = mac_cur(h);  // a launch that writes the fields calls begin_macro_write first
  a.nx = h->p.nx;
  a.ny = h->p.ny;
  a.bc = h->slab ? BC_SLAB : h->p.bc;
  a.slab_walls = h->slab ? ((h->slo ? 0 : SLAB_LO_WALL) | (h->shi ? 0 : SLAB_HI_WALL)) : 0;
  a.write_macros = write_macros;
  a.pitch = h->pitch;
  a.plane = h->plane;
  a.enc_scale = h->enc_scale;
  uint32_t* tick = reinterpret_cast<uint32_t*>(h->ws + h->off_tick);
  a.tick_in = tick + src_buf;
  a.tick_out = tick + (src_buf ^ 1);
  a.err = reinterpret_cast<int*>(tick + 2);
  if (h->p.hv_local) {
    a.um_in = h->ws + h->off_um[src_buf];
    a.um_out = h->ws + h->off_um[src_buf ^ 1];
  }
  return a;
}

cudaError_t launch_step(ltne_handle* h, int src_buf, int write_macros, cudaStream_t st,
                        bool chained = false) {
  LatticeArgs a = lattice_args(h, src_buf, write_macros);
  a.chained = chained ? 1 : 0;
  switch (h->p.storage) {
    case LTNE_F64: return launch_step_f64(a, h->P, h->shape, st);
    case LTNE_F32: return launch_step_f32(a, h->P, h->shape, st);
    case LTNE_F16DEV: return launch_step_f16(a, h->P, h->shape, st);
    default: return launch_step_bf16(a, h->P, h->shape, st);
  }
}

// Point the current macro set at the one the next write of the fields
// goes to (never the residual snapshot).
void begin_macro_write(ltne_handle* h) { h->mcur = mac_next(h); }

void drop_graphs(ltne_handle* h) {
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Capture kGraphSteps plain steps starting from buffer `parity`.
cudaError_t build_graph(ltne_handle* h, int parity) {
  cudaError_t e;
  if (!h->cap_stream) {
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  // relaxed: a launcher may query the occupancy or set a kernel attribute
  // the first time it runs, which can happen inside this capture
  e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  int b = parity;
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) {
    le = launch_step(h, b, 0, h->cap_stream, k > 0);
    b ^= 1;
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&h->graph[parity], g, 0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace

namespace ltne {

// Whether kernels may read and write the caller's host arrays directly: the
// current device reaches pageable host memory through the host's page
// tables (asked once per handle).
static bool device_reads_host_pages(ltne_handle* h) {
  if (h->direct_io < 0) {
    int dev = 0, a = 0, b = 0;
    h->direct_io = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&a, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&b, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) ==
            cudaSuccess)
      h->direct_io = (a && b) ? 1 : 0;
    cudaGetLastError();
  }
  return h->direct_io == 1;
}

static bool direct_host_io(ltne_handle* h) {
  return h->host_io != LTNE_HOST_IO_STAGED && device_reads_host_pages(h);
}

// Whether every non-null pointer is memory a kernel reaches without a
// page fault (page-locked host memory, or device or managed memory).  A
// kernel's write to a pageable page the host never touched costs a fault
// serviced by the host per page: 175 ms for the five fields of a 4096^2
// lattice into fresh arrays against 11 ms staged, so writes into pageable
// arrays are staged.
static bool all_page_locked(double* const* p, int n) {
  for (int k = 0; k < n; ++k) {
    if (!p[k]) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p[k]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost && a.type != cudaMemoryTypeDevice &&
        a.type != cudaMemoryTypeManaged)
      return false;
  }
  return true;
}

// The pinned landing place of the observables' accumulators and of one
// device word (allocated at first use, freed by ltne_destroy).
static cudaError_t ensure_pin_obs(ltne_handle* h) {
  if (h->pin_obs) return cudaSuccess;
  const cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h->pin_obs),
                                      (NACC + 1) * sizeof(double), cudaHostAllocDefault);
  if (e != cudaSuccess) h->pin_obs = nullptr;
  return e;
}

// The porosity plane from the host array through the pinned buffers: every
// value checked to lie in (0, 1) and converted to the compute type.
// INVALID_ARG on a value out of range.
static int stage_porosity(ltne_handle* h, const double* phi) {
  const int nx = h->p.nx;
  const bool dbl = h->ec == 8;
  return upload_field(h, h->ws + h->off_phi, [&](char* buf, int y0, int y1) {
    const int64_t base = (int64_t)y0 * nx, cnt = (int64_t)(y1 - y0) * nx;
    bool bad[kHostChunks] = {false};
    host_chunks(cnt, [&](int c, int64_t lo, int64_t hi) {
      for (int64_t k = lo; k < hi; ++k) {
        const double v = phi[base + k];
        if (!in_open(v, 0.0, 1.0)) {
          bad[c] = true;
          return;
        }
        if (dbl) reinterpret_cast<double*>(buf)[k] = v;
        else reinterpret_cast<float*>(buf)[k] = (float)v;
      }
    });
    for (int c = 0; c < kHostChunks; ++c)
      if (bad[c]) return false;
    return true;
  });
}

int set_fields_impl(ltne_handle* h, const double* porosity, const double* rho, const double* ux,
                    const double* uy, const double* T_f, const double* T_s, void* pre_out) {
  if (!h) return LTNE_ERR_INVALID_ARG;
  if (!h->ws) return LTNE_ERR_STATE;
  const ltne_params& p = h->p;
  if ((porosity != nullptr) != (p.porosity_field != 0)) return LTNE_ERR_INVALID_ARG;
  // The constants are checked before any device work; with a porosity field
  // the Ergun diameter waits until the field has been read below (its mean
  // formed by the porosity kernel in the direct form, on the host in the
  // staged one; any positive mean derives the same constants but the
  // diameter).
  const double any_mean = 1.0;
  int rc = derive(h, porosity ? &any_mean : nullptr);
  if (rc != LTNE_OK) return rc;
  // From here the device state is being replaced: a failure below leaves
  // the handle without fields until a set_fields call succeeds.
  h->fields_set = false;
  drop_graphs(h);  // kernel arguments captured in graphs depend on the parameters

  // Zero the whole workspace first -- population buffers, porosity, both
  // macro sets, |u| planes, counters -- so that row and plane padding, which
  // no kernel writes, is zero and state blobs are deterministic.  A lattice
  // without padding (nx a multiple of 64, nx * ny of 128) has none: every
  // element of the other planes is written before it is read, and only the
  // macro set the fields are staged into must start at zero (a field not
  // given is a zero deviation).  At 4096^2 that is 0.34 GB instead of 3 GB.
  {
    // (a slab's halo rows keep planes no step writes: always zeroed)
    const bool padded =
        h->slab || h->pitch != p.nx || h->plane != h->pitch * (int64_t)p.ny;
    const cudaError_t ez =
        padded ? cudaMemsetAsync(h->ws, 0, h->ws_bytes, h->stream)
               : cudaMemsetAsync(h->ws + h->off_mac[0], 0, 5 * (size_t)h->plane * h->ec,
                                 h->stream);
    if (ez != cudaSuccess) return fail_cuda(ez);
  }

  // Stage the given fields as deviations (rho - 1, ux, uy, T - T_ref;
  // compute type) into the macro planes, then k_init.  A field not given
  // takes its default (rho = 1, u = 0, T = T_ref), a zero deviation: the
  // zeroed plane already holds it, and nothing is staged or copied.
  const double defaults[5] = {1.0, 0.0, 0.0, p.T_ref, p.T_ref};
  const double refs[5] = {1.0, 0.0, 0.0, p.T_ref, p.T_ref};
  const double* src[5] = {rho, ux, uy, T_f, T_s};
  const bool dbl = h->ec == 8;
  const int nx = p.nx;
  // one field, rows [y0, y1), as deviations in the compute type; false if
  // any value is not finite
  auto stage = [&](const double* s, double dflt, double ref, char* dst) -> int {
    return upload_field(h, dst, [&](char* buf, int y0, int y1) {
      const int64_t base = (int64_t)y0 * nx, cnt = (int64_t)(y1 - y0) * nx;
      bool bad[kHostChunks] = {false};
      host_chunks(cnt, [&](int c, int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k) {
          const double v = (s ? s[base + k] : dflt) - ref;
          if (!isfinite(v)) bad[c] = true;
          if (dbl) reinterpret_cast<double*>(buf)[k] = v;
          else reinterpret_cast<float*>(buf)[k] = (float)v;
        }
      });
      for (int c = 0; c < kHostChunks; ++c)
        if (bad[c]) return false;
      return true;
    });
  };
  h->mcur = 0;  // the fields go to macro set 0; no residual snapshot yet
  h->msnap = -1;
  const bool erg = porosity && p.permeability == LTNE_K_ERGUN && !(p.d_p > 0) && !h->slab;
  double erg_mean = 0.0;
  if (direct_host_io(h)) {
    // kernels read the host arrays, convert and check them; the porosity
    // kernel also forms the Ergun chunk sums (the order of ergun_mean)
    HostPlanes hp;
    bool any = false;
    for (int k = 0; k < 5; ++k)
      if (src[k]) {
        hp.src[k] = src[k];
        hp.ref[k] = refs[k];
        any = true;
      }
    uint32_t* bad = reinterpret_cast<uint32_t*>(h->ws + h->off_tick) + 3;
    cudaError_t e = ensure_pin_obs(h);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), h->stream);
    if (e == cudaSuccess && any)
      e = launch_fields_from_host(mac_cur(h), dbl, h->plane, h->pitch, nx, p.ny, hp, bad,
                                  h->stream);
    // the chunk sums go to the reduction partials (room checked), then to
    // the first pinned staging buffer
    const int64_t n = (int64_t)p.nx * p.ny, chunks = ergun_chunks(n);
    const bool erg_dev = erg && (size_t)chunks <= (size_t)h->red_blocks * NACC;
    double* part = reinterpret_cast<double*>(h->ws + h->off_part);
    if (e == cudaSuccess && erg_dev) e = ensure_pinned(h, (size_t)chunks * sizeof(double));
    if (e == cudaSuccess && porosity)
      e = launch_porosity_from_host(porosity, h->ws + h->off_phi, dbl, h->pitch, nx, p.ny,
                                    erg_dev ? part : nullptr, bad, h->stream);
    uint32_t* flag = reinterpret_cast<uint32_t*>(h->pin_obs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(flag, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && erg_dev)
      e = cudaMemcpyAsync(h->pin[0], part, (size_t)chunks * sizeof(double),
                          cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(h->stream);  // no kernel may still read the caller's arrays
      return fail_cuda(e);
    }
    if (erg && !erg_dev) erg_mean = ergun_mean(porosity, n);
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail_cuda(e);
    if (*flag) return LTNE_ERR_INVALID_ARG;
    if (erg_dev) erg_mean = ergun_mean_of_chunks(reinterpret_cast<const double*>(h->pin[0]), n);
  } else {
    for (int k = 0; k < 5; ++k) {
      if (!src[k]) continue;
      rc = stage(src[k], defaults[k], refs[k], mac_cur(h) + (size_t)k * h->plane * h->ec);
      if (rc != LTNE_OK) return rc;
    }
    if (porosity) {
      rc = stage_porosity(h, porosity);
      if (rc != LTNE_OK) return rc;
      if (erg) erg_mean = ergun_mean(porosity, (int64_t)p.nx * p.ny);
    }
  }
  if (erg) {
    rc = derive(h, &erg_mean);
    if (rc != LTNE_OK) return rc;
  }
  // the step counters and the device error word start cleared
  cudaError_t e = cudaMemsetAsync(h->ws + h->off_tick, 0, 3 * sizeof(uint32_t), h->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  LatticeArgs a = lattice_args(h, 1, 1);  // dst = buffer 0
  a.pre_out = pre_out;
  switch (p.storage) {
    case LTNE_F64: e = launch_init_f64(a, h->P, h->stream); break;
    case LTNE_F32: e = launch_init_f32(a, h->P, h->stream); break;
    case LTNE_F16DEV: e = launch_init_f16(a, h->P, h->stream); break;
    default: e = launch_init_bf16(a, h->P, h->stream); break;
  }
  if (e != cudaSuccess) return fail_cuda(e);
  h->cur = 0;
  h->step = 0;
  h->fields_set = true;
  h->have_prev = false;
  return LTNE_OK;
}

int reduce_launch(ltne_handle* h) {
  const ltne_params& p = h->p;
  ReduceArgs a;
  a.mac = mac_cur(h);
  a.phi = p.porosity_field ? h->ws + h->off_phi : nullptr;
  // the snapshot's u_x, u_y, T_f, T_s planes (the current ones when there is
  // no snapshot or the fields have not changed since it: differences 0)
  a.prev = h->ws + h->off_mac[h->msnap >= 0 ? h->msnap : h->mcur] + (size_t)h->plane * h->ec;
  a.partials = reinterpret_cast<double*>(h->ws + h->off_part);
  a.out = reinterpret_cast<double*>(h->ws + h->off_out);
  a.nx = p.nx;
  a.ny = p.ny;
  a.pitch = h->pitch;
  a.plane = h->plane;
  a.phi_u = p.porosity;
  a.sigma = p.sigma;
  a.qf = p.qf;
  a.qs = p.qs;
  a.update_prev = 0;  // the snapshot is a whole macro set (see ltne_observables)
  a.blocks = h->red_blocks;
  a.is_double = h->ec == 8;
  if (h->slab) {
    // the computed rows only, with the trapezoid's half weight at a row
    // that is a wall of the whole cavity
    const size_t skip = (size_t)h->slo * h->pitch * h->ec;
    a.mac = static_cast<const char*>(a.mac) + skip;
    if (a.phi) a.phi = static_cast<const char*>(a.phi) + skip;
    a.prev = static_cast<char*>(a.prev) + skip;
    a.ny = h->srows;
    a.blocks = reduce_blocks(p.nx, h->srows);
    a.wall_lo = h->slo ? 0 : 1;
    a.wall_hi = h->shi ? 0 : 1;
  }
  return fail_cuda(launch_reduce(a, h->stream));
}

int reduce_handle(ltne_handle* h, double* acc) {
  const int rc = reduce_launch(h);
  if (rc != LTNE_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(acc, h->ws + h->off_out, NACC * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) h->msnap = h->mcur;  // these fields are the next residual's reference
  return fail_cuda(e);
}

}  // namespace ltne

// ---- row-slab decomposition on one device ---------------------------------
//
// Slab p holds rows [g0, g0 + rows) of the cavity, plus one halo row below
// (p > 0) and one above (p < nslabs - 1) with the neighbouring slabs' values;
// its first / last row is otherwise the cavity's bottom / top wall row.
namespace {

struct SlabGeom {
  int g0, rows, lo, hi;  // first global row, computed rows, halo rows below / above
  int ny;                // local rows: rows + lo + hi
  int64_t plane;         // local plane (elements)
  size_t off_pop[2], off_phi, off_mac, end;  // byte offsets in the scratch
};

std::vector<SlabGeom> slab_layout(const ltne_handle* h, int nslabs) {
  std::vector<SlabGeom> g((size_t)nslabs);
  const int ny = h->p.ny, base = ny / nslabs, extra = ny % nslabs;
  size_t off = 0;
  int y = 0;
  for (int p = 0; p < nslabs; ++p) {
    SlabGeom& s = g[(size_t)p];
    s.g0 = y;
    s.rows = base + (p < extra ? 1 : 0);
    y += s.rows;
    s.lo = p > 0;
    s.hi = p < nslabs - 1;
    s.ny = s.rows + s.lo + s.hi;
    s.plane = (int64_t)align_up((size_t)(h->pitch * s.ny), 128);
    for (int b = 0; b < 2; ++b) {
      s.off_pop[b] = off;
      off = align_up(off + 19 * (size_t)s.plane * h->es, 256);
    }
    s.off_phi = off;
    if (h->p.porosity_field) off = align_up(off + (size_t)s.plane * h->ec, 256);
    s.off_mac = off;
    off = align_up(off + 5 * (size_t)s.plane * h->ec, 256);
    s.end = off;
  }
  return g;
}

bool slabs_supported(const ltne_handle* h, int nslabs) {
  return h && !h->slab && nslabs >= 1 && h->p.bc == LTNE_BC_CAVITY && !h->p.hv_local &&
         (h->p.storage == LTNE_F32 || h->p.storage == LTNE_F64) && h->p.ny / nslabs >= 2;
}

// Copies `nrows` rows starting at src_row of `planes` planes (plane strides
// in elements, row pitch shared) between two plane sets: one 2-D copy whose
// rows are the planes' row blocks.
cudaError_t copy_rows(char* dst, int64_t dplane, int dst_row, const char* src, int64_t splane,
                      int src_row, int nrows, int planes, int64_t pitch, size_t esz,
                      cudaStream_t st) {
  const size_t w = (size_t)nrows * pitch * esz;
  return cudaMemcpy2DAsync(dst + (size_t)dst_row * pitch * esz, (size_t)dplane * esz,
                           src + (size_t)src_row * pitch * esz, (size_t)splane * esz, w,
                           (size_t)planes, cudaMemcpyDeviceToDevice, st);
}

}  // namespace

extern "C" {

void ltne_default_params(ltne_params* p, int32_t nx, int32_t ny) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->storage = LTNE_F32;
  p->bc = LTNE_BC_CAVITY;
  p->permeability = LTNE_K_DARCY;
  p->porosity_field = 0;
  p->Ra = 1e4;
  p->Pr = 1.0;
  p->Da = 1e-2;
  p->porosity = 0.6;
  p->H = 10.0;
  p->gamma_sf = 1.0;
  p->sigma = 1.0;
  p->J_e = 1.0;
  p->T_hot = 1.0;
  p->T_cold = 0.0;
  p->T_ref = 0.5;
  p->Ma = 0.1;
  p->F_phi = -1.0;
  p->d_p = 0.0;
  p->s_e = 1.1;   // Sec. 4
  p->s_eps = 1.1;
  p->s_q = 1.2;
  p->zeta_e = 1.1;
  p->zeta_nu = 1.1;
  p->eta_e = 1.1;
  p->eta_nu = 1.1;
  p->varpi = 0.4;
  p->hv_local = 0;
  p->Dp_over_L = 0.0135;  // Sec. 4
}

int ltne_create(const ltne_params* p, void* cuda_stream, ltne_handle** out) {
  if (!p || !out) return LTNE_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate_params(*p);
  if (rc != LTNE_OK) return rc;
  ltne_handle* h = new ltne_handle();
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  rc = derive(h, nullptr);
  if (rc != LTNE_OK) {
    delete h;
    return rc;
  }
  layout(h);
  // Default schedules, the fastest measured on GB300: two nodes per thread
  // in 32 x 4 blocks for 16-bit storage from 2^20 nodes up (issue-bound in
  // the one-node form: 43.5 against 42.8 GLUPS at 1024^2 FP16, 47.9 against
  // 43.5 at 2048^2; 35.1 against 38.6 at 724^2), in 128 x 1
  // blocks for FP32 from 2^22 nodes up (at the HBM roofline either way;
  // below, one node per thread is faster: 39.5 against 37.3 GLUPS at
  // 1024^2, equal at 2048^2); one node per thread in 64 x 2 blocks for FP64
  // and for smaller lattices, whose steps are a single wave or a few, bound
  // by the latency of one thread's work (64 x 2 against 128 x 2: 40.5
  // against 38.3 GLUPS at 512^2 FP32, 34.2 against 32.2 FP16, equal at
  // 256^2 and in FP64).
  const int64_t nodes = (int64_t)p->nx * p->ny;
  if ((p->storage == LTNE_F16DEV || p->storage == LTNE_BF16DEV) && nodes >= ((int64_t)1 << 20)) {
    h->shape.bx = 32;
    h->shape.by = 4;
    h->shape.pair = 1;
  } else if (p->storage == LTNE_F32 && nodes >= ((int64_t)1 << 22)) {
    h->shape.bx = 128;
    h->shape.by = 1;
    h->shape.pair = 1;
  }
  *out = h;
  return LTNE_OK;
}

size_t ltne_workspace_bytes(const ltne_handle* h) { return h ? h->ws_bytes : 0; }

int ltne_bind_workspace(ltne_handle* h, void* device_ptr, size_t bytes) {
  if (!h || !device_ptr) return LTNE_ERR_INVALID_ARG;
  if (bytes < h->ws_bytes || (reinterpret_cast<uintptr_t>(device_ptr) & 255u) != 0)
    return LTNE_ERR_WORKSPACE;
  drop_graphs(h);
  h->ws = static_cast<char*>(device_ptr);
  h->fields_set = false;
  return LTNE_OK;
}

int ltne_set_fields(ltne_handle* h, const double* porosity, const double* rho, const double* ux,
                    const double* uy, const double* T_f, const double* T_s) {
  return set_fields_impl(h, porosity, rho, ux, uy, T_f, T_s, nullptr);
}

int ltne_step(ltne_handle* h, int64_t n) {
  if (!h || n < 0 || h->slab) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  if (n == 0) return LTNE_OK;
  int64_t plain = n - 1;  // the last step also writes the macroscopic fields
  cudaError_t e;
  while (plain >= kGraphSteps) {
    if (!h->graph[h->cur]) {
      e = build_graph(h, h->cur);
      if (e != cudaSuccess) return fail_cuda(e);
    }
    e = cudaGraphLaunch(h->graph[h->cur], h->stream);
    if (e != cudaSuccess) return fail_cuda(e);
    plain -= kGraphSteps;
    h->step += kGraphSteps;
    h->launches += kGraphSteps;
  }
  bool chained = false;  // the stream's last operation is a step kernel of this call
  for (; plain > 0; --plain) {
    e = launch_step(h, h->cur, 0, h->stream, chained);
    if (e != cudaSuccess) return fail_cuda(e);
    chained = true;
    h->cur ^= 1;
    ++h->step;
    ++h->launches;
  }
  begin_macro_write(h);  // the last step writes the fields
  e = launch_step(h, h->cur, 1, h->stream, chained);
  if (e != cudaSuccess) return fail_cuda(e);
  h->cur ^= 1;
  ++h->step;
  ++h->launches;
  return LTNE_OK;
}

int ltne_observables(ltne_handle* h, ltne_obs* out) {
  if (!h || !out || h->slab) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  const ltne_params& p = h->p;
  cudaError_t e = cudaSuccess;
  e = ensure_pin_obs(h);
  if (e != cudaSuccess) return fail_cuda(e);
  const int rr = reduce_launch(h);
  if (rr != LTNE_OK) return rr;
  // the accumulators and the device error word in one read-back: a staged
  // step that gave up waiting for its tile reports here (the fields are then
  // not trustworthy); the word is cleared
  int* errp = reinterpret_cast<int*>(h->pin_obs + NACC);
  e = cudaMemcpyAsync(h->pin_obs, h->ws + h->off_out, NACC * sizeof(double),
                      cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(errp, h->ws + h->off_tick + 2 * sizeof(uint32_t), sizeof(int),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  double acc[NACC];
  for (int k = 0; k < NACC; ++k) acc[k] = h->pin_obs[k];
  const int err = *errp;
  if (err) {
    e = cudaMemsetAsync(h->ws + h->off_tick + 2 * sizeof(uint32_t), 0, sizeof(err), h->stream);
    return e == cudaSuccess ? LTNE_ERR_TIMEOUT : fail_cuda(e);
  }
  DerivedInfo info;
  info.L = h->L;
  info.nu_f = h->nu_f;
  info.alpha_f = h->alpha_f;
  const int rc = finish_observables(p, info, h->step, h->msnap >= 0, acc, out);
  h->have_prev = true;
  h->msnap = h->mcur;  // these fields are the next residual's reference
  return rc;
}

int ltne_get_fields(ltne_handle* h, double* rho, double* ux, double* uy, double* T_f, double* T_s) {
  if (!h) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  const ltne_params& p = h->p;
  double* dst[5] = {rho, ux, uy, T_f, T_s};
  const int nx = p.nx;
  if (direct_host_io(h) && all_page_locked(dst, 5)) {  // one kernel writes the caller's arrays
    HostPlanes hp;
    for (int k = 0; k < 5; ++k) {
      hp.dst[k] = dst[k];
      hp.ref[k] = (k == 0) ? 1.0 : (k >= 3 ? p.T_ref : 0.0);  // planes hold deviations
    }
    cudaError_t e = launch_fields_to_host(mac_cur(h), h->ec == 8, h->plane, h->pitch, nx, p.ny,
                                          hp, h->stream);
    const cudaError_t es = cudaStreamSynchronize(h->stream);
    return fail_cuda(e != cudaSuccess ? e : es);
  }
  for (int k = 0; k < 5; ++k) {
    if (!dst[k]) continue;
    const double ref = (k == 0) ? 1.0 : (k >= 3 ? p.T_ref : 0.0);  // planes hold deviations
    double* out = dst[k];
    const int rc = download_field(
        h, mac_cur(h) + (size_t)k * h->plane * h->ec, [&](const char* buf, int y0, int y1) {
          const int64_t base = (int64_t)y0 * nx, cnt = (int64_t)(y1 - y0) * nx;
          if (h->ec == 8) {
            const double* t = reinterpret_cast<const double*>(buf);
            host_chunks(cnt, [&](int, int64_t lo, int64_t hi) {
              for (int64_t i = lo; i < hi; ++i) out[base + i] = ref + t[i];
            });
          } else {
            const float* t = reinterpret_cast<const float*>(buf);
            host_chunks(cnt, [&](int, int64_t lo, int64_t hi) {
              for (int64_t i = lo; i < hi; ++i) out[base + i] = ref + (double)t[i];
            });
          }
        });
    if (rc != LTNE_OK) return rc;
  }
  return LTNE_OK;
}

// State blob: 64-byte header (magic, storage, nx, ny, step, plane, Ergun
// diameter in use), then in the device layout the current populations (19
// planes), the macroscopic planes (5), the |u| plane of the local h_v model
// (if on) and the porosity plane (if per node).
size_t ltne_state_bytes(const ltne_handle* h) {
  if (!h) return 0;
  return 64 + 19 * (size_t)h->plane * h->es + 5 * (size_t)h->plane * h->ec +
         (h->p.hv_local ? (size_t)h->plane * h->ec : 0) +
         (h->p.porosity_field ? (size_t)h->plane * h->ec : 0);
}

int ltne_get_state(ltne_handle* h, void* host, size_t bytes) {
  if (!h || !host || bytes < ltne_state_bytes(h)) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  uint64_t dbits = 0;  // the Ergun diameter in use travels with the porosity
  memcpy(&dbits, &h->d_ergun, sizeof(dbits));
  uint64_t hdr[8] = {kStateMagic, (uint64_t)h->p.storage, (uint64_t)h->p.nx,
                     (uint64_t)h->p.ny, (uint64_t)h->step, (uint64_t)h->plane, dbits, 0};
  memcpy(host, hdr, sizeof(hdr));
  char* dst = static_cast<char*>(host) + 64;
  const size_t pb = 19 * (size_t)h->plane * h->es, mb = 5 * (size_t)h->plane * h->ec;
  cudaError_t e = cudaMemcpyAsync(dst, h->ws + h->off_pop[h->cur], pb, cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + pb, mac_cur(h), mb, cudaMemcpyDeviceToHost, h->stream);
  const size_t ub = h->p.hv_local ? (size_t)h->plane * h->ec : 0;
  if (e == cudaSuccess && ub)
    e = cudaMemcpyAsync(dst + pb + mb, h->ws + h->off_um[h->cur], ub, cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess && h->p.porosity_field)
    e = cudaMemcpyAsync(dst + pb + mb + ub, h->ws + h->off_phi, (size_t)h->plane * h->ec,
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return fail_cuda(e);
}

int ltne_set_state(ltne_handle* h, const void* host, size_t bytes) {
  if (!h || !host || bytes < ltne_state_bytes(h)) return LTNE_ERR_INVALID_ARG;
  if (!h->ws) return LTNE_ERR_STATE;
  uint64_t hdr[8];
  memcpy(hdr, host, sizeof(hdr));
  if (hdr[0] != kStateMagic || hdr[1] != (uint64_t)h->p.storage || hdr[2] != (uint64_t)h->p.nx ||
      hdr[3] != (uint64_t)h->p.ny || hdr[5] != (uint64_t)h->plane)
    return LTNE_ERR_INVALID_ARG;
  const char* src = static_cast<const char*>(host) + 64;
  const size_t pb = 19 * (size_t)h->plane * h->es, mb = 5 * (size_t)h->plane * h->ec;
  h->mcur = 0;  // the restored fields in macro set 0; no residual snapshot
  h->msnap = -1;
  cudaError_t e = cudaMemcpyAsync(h->ws + h->off_pop[0], src, pb, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mac_cur(h), src + pb, mb, cudaMemcpyHostToDevice, h->stream);
  const size_t ub = h->p.hv_local ? (size_t)h->plane * h->ec : 0;
  if (e == cudaSuccess && ub)
    e = cudaMemcpyAsync(h->ws + h->off_um[0], src + pb + mb, ub, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess && h->p.porosity_field) {
    e = cudaMemcpyAsync(h->ws + h->off_phi, src + pb + mb + ub, (size_t)h->plane * h->ec,
                        cudaMemcpyHostToDevice, h->stream);
    // the lattice constants that depend on the porosity field: the Ergun
    // diameter is taken from the checkpoint, not re-derived
    double d = 0.0;
    memcpy(&d, &hdr[6], sizeof(d));
    if (h->p.permeability == LTNE_K_ERGUN && h->p.d_p <= 0 && d > 0) {
      h->p.d_p = d;
      const int rc = derive(h, nullptr);
      if (rc != LTNE_OK) return rc;
      drop_graphs(h);
    }
  }
  // the rounding stream is keyed by the step; the other counter slot and
  // the device error word start cleared
  const uint32_t words[3] = {(uint32_t)hdr[4], 0u, 0u};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + h->off_tick, words, sizeof(words), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  h->cur = 0;
  h->step = (int64_t)hdr[4];
  h->fields_set = true;
  h->have_prev = false;
  return LTNE_OK;
}

int64_t ltne_launch_count(const ltne_handle* h) { return h ? h->launches : 0; }

int ltne_set_schedule(ltne_handle* h, int32_t block_x, int32_t block_y,
                      int32_t nodes_per_thread) {
  if (!h) return LTNE_ERR_INVALID_ARG;
  const int64_t threads = (int64_t)block_x * block_y;
  if (block_x < 32 || block_x > 256 || block_x % 32 != 0 || block_y < 1 || threads > 256)
    return LTNE_ERR_INVALID_ARG;
  if (nodes_per_thread != 1 && nodes_per_thread != 2) return LTNE_ERR_INVALID_ARG;
  if (nodes_per_thread == 2 &&
      (h->p.storage == LTNE_F64 || threads > kPairBlockThreads || h->slab))
    return LTNE_ERR_INVALID_ARG;
  h->shape.bx = block_x;
  h->shape.by = block_y;
  h->shape.pair = nodes_per_thread == 2 ? 1 : 0;
  drop_graphs(h);  // the captured launches carry the old configuration
  return LTNE_OK;
}

size_t ltne_slab_scratch_bytes(const ltne_handle* h, int32_t nslabs) {
  if (!slabs_supported(h, nslabs)) return 0;
  return slab_layout(h, nslabs).back().end;
}

int ltne_step_slabs(ltne_handle* h, int32_t nslabs, int64_t n, void* scratch, size_t bytes) {
  if (!slabs_supported(h, nslabs) || n < 0) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  const std::vector<SlabGeom> g = slab_layout(h, nslabs);
  char* ws = static_cast<char*>(scratch);
  if (!ws || bytes < g.back().end || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return LTNE_ERR_WORKSPACE;
  if (n == 0) return LTNE_OK;
  const int64_t pitch = h->pitch;
  const size_t es = h->es, ec = h->ec;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  // zeroed slab buffers keep the row padding of the gathered planes zero (as
  // in the handle), then scatter the current populations (halo rows
  // included) and the porosity
  e = cudaMemsetAsync(ws, 0, g.back().end, st);
  if (e != cudaSuccess) return fail_cuda(e);
  for (const SlabGeom& s : g) {
    e = copy_rows(ws + s.off_pop[0], s.plane, 0, h->ws + h->off_pop[h->cur], h->plane,
                  s.g0 - s.lo, s.ny, 19, pitch, es, st);
    if (e == cudaSuccess && h->p.porosity_field)
      e = copy_rows(ws + s.off_phi, s.plane, 0, h->ws + h->off_phi, h->plane, s.g0 - s.lo, s.ny,
                    1, pitch, ec, st);
    if (e != cudaSuccess) return fail_cuda(e);
  }
  StepShape one;  // one node per thread, 64 x 2
  int b = 0;
  for (int64_t k = 0; k < n && e == cudaSuccess; ++k) {
    for (const SlabGeom& s : g) {
      LatticeArgs a = lattice_args(h, h->cur, k == n - 1 ? 1 : 0);
      a.src = ws + s.off_pop[b];
      a.dst = ws + s.off_pop[b ^ 1];
      a.phi = h->p.porosity_field ? ws + s.off_phi : nullptr;
      a.mac = ws + s.off_mac;
      a.ny = s.ny;
      a.plane = s.plane;
      a.bc = BC_SLAB;
      a.slab_walls = (s.lo ? 0 : SLAB_LO_WALL) | (s.hi ? 0 : SLAB_HI_WALL);
      e = h->p.storage == LTNE_F64 ? launch_step_f64(a, h->P, one, st)
                                   : launch_step_f32(a, h->P, one, st);
      if (e != cudaSuccess) break;
    }
    // halo exchange across every cut: the lower slab's last computed row to
    // the upper slab's halo below, the upper slab's first to the lower's halo above
    for (int p = 0; p + 1 < nslabs && e == cudaSuccess; ++p) {
      const SlabGeom &lo = g[(size_t)p], &up = g[(size_t)p + 1];
      e = copy_rows(ws + up.off_pop[b ^ 1], up.plane, 0, ws + lo.off_pop[b ^ 1], lo.plane,
                    lo.lo + lo.rows - 1, 1, 19, pitch, es, st);
      if (e == cudaSuccess)
        e = copy_rows(ws + lo.off_pop[b ^ 1], lo.plane, lo.ny - 1, ws + up.off_pop[b ^ 1],
                      up.plane, up.lo, 1, 19, pitch, es, st);
    }
    b ^= 1;
  }
  if (e != cudaSuccess) return fail_cuda(e);
  // gather the computed rows and the macroscopic fields of the last step
  const int out = h->cur ^ (int)(n & 1);
  begin_macro_write(h);
  for (const SlabGeom& s : g) {
    e = copy_rows(h->ws + h->off_pop[out], h->plane, s.g0, ws + s.off_pop[b], s.plane, s.lo,
                  s.rows, 19, pitch, es, st);
    if (e == cudaSuccess)
      e = copy_rows(mac_cur(h), h->plane, s.g0, ws + s.off_mac, s.plane, s.lo, s.rows, 5,
                    pitch, ec, st);
    if (e != cudaSuccess) return fail_cuda(e);
  }
  h->cur = out;
  h->step += n;
  h->launches += n * nslabs;
  return LTNE_OK;
}

// ---- a row slab per process ------------------------------------------------

int ltne_slab_rows(int32_t ny, int32_t nslabs, int32_t index, int32_t* y0, int32_t* rows,
                   int32_t* halo_lo, int32_t* halo_hi) {
  if (ny < 4 || nslabs < 1 || index < 0 || index >= nslabs || ny / nslabs < 2)
    return LTNE_ERR_INVALID_ARG;
  const int base = ny / nslabs, extra = ny % nslabs;
  if (y0) *y0 = index * base + std::min(index, extra);
  if (rows) *rows = base + (index < extra ? 1 : 0);
  if (halo_lo) *halo_lo = index > 0 ? 1 : 0;
  if (halo_hi) *halo_hi = index < nslabs - 1 ? 1 : 0;
  return LTNE_OK;
}

int ltne_create_slab(const ltne_params* p, int32_t nslabs, int32_t index, void* cuda_stream,
                     ltne_handle** out) {
  if (!p || !out) return LTNE_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate_params(*p);
  if (rc != LTNE_OK) return rc;
  if (p->bc != LTNE_BC_CAVITY || p->hv_local ||
      (p->storage != LTNE_F32 && p->storage != LTNE_F64))
    return LTNE_ERR_INVALID_ARG;
  // the Ergun diameter belongs to the whole porosity field, which no slab sees
  if (p->permeability == LTNE_K_ERGUN && p->porosity_field && !(p->d_p > 0))
    return LTNE_ERR_INVALID_ARG;
  int32_t y0 = 0, rows = 0, lo = 0, hi = 0;
  rc = ltne_slab_rows(p->ny, nslabs, index, &y0, &rows, &lo, &hi);
  if (rc != LTNE_OK) return rc;
  ltne_handle* h = new ltne_handle();
  h->p = *p;
  h->slab = 1;
  h->nslabs = nslabs;
  h->slab_index = index;
  h->gny = p->ny;
  h->g0 = y0;
  h->srows = rows;
  h->slo = lo;
  h->shi = hi;
  h->p.ny = rows + lo + hi;  // the local lattice
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  rc = derive(h, nullptr);
  if (rc != LTNE_OK) {
    delete h;
    return rc;
  }
  layout(h);  // one node per thread, 64 x 2 blocks (the slab kernel's form)
  *out = h;
  return LTNE_OK;
}

int ltne_halo_buffers(ltne_handle* h, void** send_lo, void** send_hi, void** recv_lo,
                      void** recv_hi, size_t* bytes) {
  if (!h || !h->slab) return LTNE_ERR_INVALID_ARG;
  if (!h->ws) return LTNE_ERR_STATE;
  void* ptr[4];
  for (int k = 0; k < 4; ++k) {
    const bool has = (k & 1) ? h->shi : h->slo;
    ptr[k] = has ? h->ws + h->off_halo[k] : nullptr;
  }
  if (send_lo) *send_lo = ptr[0];
  if (send_hi) *send_hi = ptr[1];
  if (recv_lo) *recv_lo = ptr[2];
  if (recv_hi) *recv_hi = ptr[3];
  if (bytes) *bytes = 5 * (size_t)h->p.nx * h->es;
  return LTNE_OK;
}

int ltne_halo_pack(ltne_handle* h) {
  if (!h || !h->slab) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  return fail_cuda(launch_halo_pack(h->ws + h->off_pop[h->cur], h->pitch, h->plane, h->p.nx,
                                    h->slo, h->slo + h->srows - 1, h->es,
                                    h->slo ? h->ws + h->off_halo[0] : nullptr,
                                    h->shi ? h->ws + h->off_halo[1] : nullptr, h->stream));
}

int ltne_halo_unpack(ltne_handle* h) {
  if (!h || !h->slab) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  return fail_cuda(launch_halo_unpack(h->ws + h->off_pop[h->cur], h->pitch, h->plane, h->p.nx,
                                      0, h->p.ny - 1, h->es,
                                      h->slo ? h->ws + h->off_halo[2] : nullptr,
                                      h->shi ? h->ws + h->off_halo[3] : nullptr, h->stream));
}

int ltne_step_slab(ltne_handle* h, int32_t write_macros) {
  if (!h || !h->slab || (write_macros != 0 && write_macros != 1)) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  if (write_macros) begin_macro_write(h);
  const cudaError_t e = launch_step(h, h->cur, write_macros, h->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  h->cur ^= 1;
  ++h->step;
  ++h->launches;
  return ltne_halo_pack(h);
}

int ltne_slab_accumulators(ltne_handle* h, double* acc, int32_t nacc) {
  if (!h || !h->slab || !acc || nacc != NACC) return LTNE_ERR_INVALID_ARG;
  if (!h->ws || !h->fields_set) return LTNE_ERR_STATE;
  return reduce_handle(h, acc);
}

int ltne_accumulators_combine(double* acc, const double* other, int32_t nacc) {
  if (!acc || !other || nacc != NACC) return LTNE_ERR_INVALID_ARG;
  for (int k = 0; k < NACC; ++k)
    acc[k] = (k == A_MAXU || k == A_MAXDT) ? fmax(acc[k], other[k]) : acc[k] + other[k];
  return LTNE_OK;
}

int ltne_observables_from_accumulators(const ltne_params* p, int64_t step, int32_t have_prev,
                                       const double* acc, int32_t nacc, ltne_obs* out) {
  if (!p || !acc || !out || nacc != NACC) return LTNE_ERR_INVALID_ARG;
  int rc = validate_params(*p);
  if (rc != LTNE_OK) return rc;
  NodeParams<double> P;
  DerivedInfo info;
  ltne_params q = *p;
  if (q.permeability == LTNE_K_ERGUN && q.porosity_field && !(q.d_p > 0)) q.d_p = 1.0;
  rc = derive_params(q, nullptr, P, info);  // L and alpha_f (no diameter is needed)
  if (rc != LTNE_OK) return rc;
  return finish_observables(*p, info, step, have_prev != 0, acc, out);
}

int ltne_ergun_diameter(const double* porosity, int64_t n, double L, double Da, double* d) {
  if (!porosity || n < 1 || !d || !(L > 0) || !(Da > 0)) return LTNE_ERR_INVALID_ARG;
  bool bad[kHostChunks] = {false};
  host_chunks(n, [&](int c, int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi && !bad[c]; ++k) bad[c] = !in_open(porosity[k], 0.0, 1.0);
  });
  for (int c = 0; c < kHostChunks; ++c)
    if (bad[c]) return LTNE_ERR_INVALID_ARG;
  *d = L * sqrt(150.0 * Da / ergun_mean(porosity, n));
  return LTNE_OK;
}

int ltne_set_host_io(ltne_handle* h, int32_t mode) {
  if (!h || mode < LTNE_HOST_IO_AUTO || mode > LTNE_HOST_IO_DIRECT) return LTNE_ERR_INVALID_ARG;
  if (mode == LTNE_HOST_IO_DIRECT && !device_reads_host_pages(h)) return LTNE_ERR_INVALID_ARG;
  h->host_io = mode;
  return LTNE_OK;
}

int ltne_get_host_io(ltne_handle* h, int32_t* mode) {
  if (!h || !mode) return LTNE_ERR_INVALID_ARG;
  *mode = direct_host_io(h) ? LTNE_HOST_IO_DIRECT : LTNE_HOST_IO_STAGED;
  return LTNE_OK;
}

int ltne_set_staging(ltne_handle* h, int32_t staged) {
  if (!h || (staged != 0 && staged != 1) || (staged && h->slab)) return LTNE_ERR_INVALID_ARG;
  if (staged && (h->p.storage == LTNE_F64 || h->p.bc != LTNE_BC_CAVITY))
    return LTNE_ERR_INVALID_ARG;
  h->shape.tma = staged;
  drop_graphs(h);
  return LTNE_OK;
}

int ltne_get_staging(const ltne_handle* h, int32_t* staged) {
  if (!h || !staged) return LTNE_ERR_INVALID_ARG;
  *staged = h->shape.tma;
  return LTNE_OK;
}

int ltne_get_schedule(const ltne_handle* h, int32_t* block_x, int32_t* block_y,
                      int32_t* nodes_per_thread) {
  if (!h || !block_x || !block_y || !nodes_per_thread) return LTNE_ERR_INVALID_ARG;
  *block_x = h->shape.bx;
  *block_y = h->shape.by;
  *nodes_per_thread = h->shape.pair ? 2 : 1;
  return LTNE_OK;
}

void ltne_destroy(ltne_handle* h) {
  if (!h) return;
  drop_graphs(h);
  release_pinned(h);
  if (h->pin_obs) cudaFreeHost(h->pin_obs);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  delete h;
}

const char* ltne_error_string(int code) {
  switch (code) {
    case LTNE_OK: return "LTNE_OK";
    case LTNE_ERR_INVALID_ARG: return "LTNE_ERR_INVALID_ARG: invalid argument or parameter";
    case LTNE_ERR_UNSTABLE_TAU: return "LTNE_ERR_UNSTABLE_TAU: a relaxation rate is outside (0, 2)";
    case LTNE_ERR_CUDA: return "LTNE_ERR_CUDA: a CUDA runtime call failed";
    case LTNE_ERR_NONFINITE: return "LTNE_ERR_NONFINITE: non-finite values in the fields";
    case LTNE_ERR_TIMEOUT: return "LTNE_ERR_TIMEOUT: a bounded device wait gave up";
    case LTNE_ERR_STATE: return "LTNE_ERR_STATE: call out of order";
    case LTNE_ERR_WORKSPACE: return "LTNE_ERR_WORKSPACE: workspace missing, too small or misaligned";
    default: return "LTNE_ERR_UNKNOWN";
  }
}

}  // extern "C"
