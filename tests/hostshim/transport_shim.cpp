// Host build of the transport kernels' per-packet code (transport.cuh: launch_packet, step and what they
// call) in FP32 or FP64, for CPU tests against the oracle: packets run one after another, as one lane of a
// single-disk kernel runs them, over a model built by the library's own host builders (tables.h).
// Compiled by the host compiler with the single-lane stand-ins of cuda_host_stubs.h.
#include "cuda_host_stubs.h"
#include "tables.h"
#include "transport.cuh"

using namespace mcrt;

namespace {

template <class R, bool G, bool POL, bool JT>
void run_packets(const KParams<R>& P, const DevModel<R>& M, uint64_t n, Acc& acc) {
  for (uint64_t k = 0; k < n; ++k) {
    Pkt<R> s;
    std::memset(&s, 0, sizeof(s));
    SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
    launch_packet<R, false, G, POL, JT>(P, rng, M, s, k, -1, acc);
    while (step<R, false, G, POL, JT>(P, rng, M, s, acc)) {
    }
  }
}

// Packets 0 .. n-1 with up to `lanes` of them in flight at once: one step of every packet in flight per
// round, a finished packet's slot refilled with the next id -- the order in which a persistent kernel's
// lanes interleave their packets' events, here one after another on one thread.
template <class R, bool G>
void run_interleaved(const KParams<R>& P, const DevModel<R>& M, uint64_t n, uint64_t lanes, Acc& acc) {
  std::vector<Pkt<R>> st(lanes);
  std::vector<char> act(lanes, 0);
  SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
  uint64_t next = 0, live = 0;
  for (uint64_t l = 0; l < lanes && next < n; ++l) {
    std::memset(&st[l], 0, sizeof(Pkt<R>));
    launch_packet<R, false, G>(P, rng, M, st[l], next++, -1, acc);
    act[l] = 1;
    ++live;
  }
  while (live) {
    for (uint64_t l = 0; l < lanes; ++l) {
      if (!act[l]) continue;
      if (!step<R, false, G>(P, rng, M, st[l], acc)) {
        if (next < n) {
          std::memset(&st[l], 0, sizeof(Pkt<R>));
          launch_packet<R, false, G>(P, rng, M, st[l], next++, -1, acc);
        } else {
          act[l] = 0;
          --live;
        }
      }
    }
  }
}

template <class R>
std::vector<R> cast(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

struct Inputs {
  int nr, nt, nlam;
  const double *rf_cm, *tf, *rho, *lam_e, *kabs, *ksca, *g;
  double Tstar, Rstar;
  uint64_t n, seed;
  int mrw, nmin, want_sed, nmu;
  double gamma;
  const double* mueller;  // [nlam][4][nmu] or NULL
  const double* Lsrc;     // internal sources: luminosity per cell (erg/s), or NULL
  uint64_t lanes;         // > 0: packets in flight at once (run_interleaved), 0: one after another
  // replay instead of packets: {ir, itheta, px, py, pz, ux, uy, uz, tau, xcross, max_calls} (positions in
  // units of the inner radius; the values of the recorded state), or NULL
  const double* replay;
};

struct Outputs {
  uint64_t *tally, *visits, *nabs, *sed, *sed_q, *sed_u, *counters;
  double* jlen;
  int64_t* replay_out;  // {advance calls, face crossings, last result, error flags, ir, itheta}
};

// Moves one gray packet from a given state with advance() alone (no interaction is run): until it reaches
// an interaction point, ends, or max_calls calls. This replays the geometry of a recorded state.
template <class R, bool G>
void replay_advance(const KParams<R>& P, const DevModel<R>& M, const double* st, int64_t* out) {
  Pkt<R> s;
  std::memset(&s, 0, sizeof(s));
  s.ir = (int)st[0];
  s.it = (int)st[1];
  s.px = (R)st[2];
  s.py = (R)st[3];
  s.pz = (R)st[4];
  s.ux = (R)st[5];
  s.uy = (R)st[6];
  s.uz = (R)st[7];
  s.tau = (R)st[8];
  s.xcross = (unsigned)st[9];
  s.plo = 1u;
  if (s.ir >= 0) set_alpha<R, G>(M, s);
  SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
  Acc acc;
  std::memset(&acc, 0, sizeof(acc));
  const int64_t max_calls = (int64_t)st[10];
  int64_t calls = 0;
  int r = 1;
  while (calls < max_calls) {
    r = advance<R, false, G, false, false>(P, rng, M, s, acc);
    ++calls;
    if (r != 1) break;
  }
  out[0] = calls;
  out[1] = acc.cross;
  out[2] = r;
  out[3] = acc.err;
  out[4] = s.ir;
  out[5] = s.it;
}

// the model as the library builds it (make_model, fill_params), in precision R
template <class R>
void run(const Inputs& in, const Outputs& out) {
  const int nr = in.nr, nt = in.nt, nlam = in.nlam;
  GeomArrays geo;
  geometry_arrays(nr, nt, in.rf_cm, in.tf, geo);
  DensityArrays den;
  density_arrays(nr, nt, in.rf_cm, in.tf, in.rho, den);
  DustArrays dust;
  dust_arrays(nlam, in.lam_e, in.kabs, in.ksca, in.g, in.Tstar, dust);
  const int nT = 1024;
  TGridTables tt;
  build_T_tables(nlam, in.lam_e, in.kabs, dust.chip.data(), nT, 1.0, std::max(1e4, 2.0 * in.Tstar), tt);
  std::vector<float> mtab(2 * kMrwTab);
  build_mrw_table(mtab.data());
  std::vector<double> gq(in.g, in.g + nlam), mt, mc;
  if (in.mueller) {
    mt.assign(in.mueller, in.mueller + (size_t)nlam * 4 * in.nmu);
    mc.resize((size_t)nlam * in.nmu);
    for (int b = 0; b < nlam; ++b) mueller_cdf(in.mueller + (size_t)b * 4 * in.nmu, in.nmu, mc.data() + (size_t)b * in.nmu);
  }
  bool gray = true;
  for (int b = 1; b < nlam; ++b)
    if (in.kabs[b] != in.kabs[0] || in.ksca[b] != in.ksca[0] || in.g[b] != in.g[0]) gray = false;
  std::vector<unsigned long long> cnt(C_NCNT, 0ull);
  // internal sources as mcrt_set_sources keeps them: cumulative luminosity in cell order
  const size_t ncell = (size_t)nr * nt;
  std::vector<double> src_cum(ncell + 1, 0.0);
  if (in.Lsrc)
    for (size_t c = 0; c < ncell; ++c) src_cum[c + 1] = src_cum[c] + in.Lsrc[c];
  const double Lsrc = src_cum[ncell];
  const std::vector<R> rf = cast<R>(geo.rf), rf2 = cast<R>(geo.rf2), c2 = cast<R>(geo.c2), s2 = cast<R>(geo.s2),
                       cf = cast<R>(geo.cf), sf = cast<R>(geo.sf), rho = cast<R>(den.rhol), chi = cast<R>(dust.chi),
                       alb = cast<R>(dust.alb), g = cast<R>(gq), star = cast<R>(dust.star), mtr = cast<R>(mt),
                       mcr = cast<R>(mc);

  DevModel<R> M;
  std::memset(&M, 0, sizeof(M));
  M.nr = nr;
  M.nt = nt;
  M.nlam = nlam;
  M.nT = nT;
  M.gray = gray ? 1 : 0;
  M.rf = rf.data();
  M.rf2 = rf2.data();
  M.c2 = c2.data();
  M.s2 = s2.data();
  M.cf = cf.data();
  M.sf = sf.data();
  M.fk = geo.fk.data();
  M.rho = rho.data();
  M.chi = chi.data();
  M.alb = alb.data();
  M.gq = g.data();
  M.star_cum = star.data();
  const double chi0 = in.kabs[0] + in.ksca[0];
  M.chi0 = (R)chi0;
  M.alb0 = (R)(in.ksca[0] / chi0);
  M.g0 = (R)in.g[0];
  M.chiR0 = (R)(in.kabs[0] + (1.0 - in.g[0]) * in.ksca[0]);
  M.kbar0 = (R)in.kabs[0];
  M.lQk = tt.lQk.data();
  M.cbw = tt.cbw.data();
  M.cexit = tt.cexit.data();
  M.chiR = tt.chiRk.data();
  M.kbar = tt.kbark.data();
  M.lqm = den.lqm.data();
  const double Lstar = 4.0 * kPi * in.Rstar * in.Rstar * MCRT_SIGMA * std::pow(in.Tstar, 4);
  M.lq_run = (float)std::log((Lstar + Lsrc) / ((double)in.n * (double)kEUnit));
  M.src_cum = Lsrc > 0 ? src_cum.data() : nullptr;
  M.src_Lstar = Lstar;
  M.src_Ltot = Lstar + Lsrc;
  M.n_src = Lsrc > 0 ? (int)ncell : 0;
  M.mtab = in.mueller ? mtr.data() : nullptr;
  M.mcdf = in.mueller ? mcr.data() : nullptr;
  M.nmu = in.mueller ? in.nmu : 0;
  M.sed_q = (unsigned long long*)out.sed_q;
  M.sed_u = (unsigned long long*)out.sed_u;
  M.jlen = out.jlen;
  M.jw = tt.jw.data();
  M.tally = (unsigned long long*)out.tally;
  M.visits = (unsigned long long*)out.visits;
  M.nabs = (unsigned long long*)out.nabs;
  M.sed = (unsigned long long*)out.sed;
  M.cnt = cnt.data();
  M.n_packets = in.n;

  KParams<R> P;
  std::memset(&P, 0, sizeof(P));
  P.m0 = M;
  P.mrw = in.mrw ? 1 : 0;
  P.nmin = in.nmin;
  P.exit_dir = 0;
  P.want_lam = (!gray || in.want_sed) ? 1 : 0;
  P.refill = 4;
  P.defer = 8;
  P.gamma = (R)in.gamma;
  P.seed = in.seed;
  P.max_events = 1ull << 31;
  P.max_steps = 4000000000ull;
  P.mrw_tab = mtab.data();
  P.mrw_t0 = mrw_table_t0();
  P.mrw_dt = mrw_table_dt();
  P.nmodels = 1;

  if (in.replay) {
    if (gray) replay_advance<R, true>(P, M, in.replay, out.replay_out);
    else replay_advance<R, false>(P, M, in.replay, out.replay_out);
    return;
  }
  Acc acc;
  std::memset(&acc, 0, sizeof(acc));
  const bool pol = in.mueller != nullptr, jt = out.jlen != nullptr;
  if (pol) {
    if (gray) run_packets<R, true, true, false>(P, M, in.n, acc);
    else run_packets<R, false, true, false>(P, M, in.n, acc);
  } else if (jt) {
    if (gray) run_packets<R, true, false, true>(P, M, in.n, acc);
    else run_packets<R, false, false, true>(P, M, in.n, acc);
  } else if (in.lanes) {
    if (gray) run_interleaved<R, true>(P, M, in.n, in.lanes, acc);
    else run_interleaved<R, false>(P, M, in.n, in.lanes, acc);
  } else {
    if (gray) run_packets<R, true, false, false>(P, M, in.n, acc);
    else run_packets<R, false, false, false>(P, M, in.n, acc);
  }
  const unsigned long long c[8] = {acc.packets, acc.abs, acc.sca, acc.cross, acc.mrw, acc.capped, acc.escaped, acc.err};
  for (int i = 0; i < 8; ++i) out.counters[i] = c[i];
}

}  // namespace

// Transports packets 0 .. n-1 with Philox key `seed` through the disk (cgs inputs, as mcrt_disk_create and
// mcrt_set_opacity take them), in FP32 (prec 32) or FP64, polarized with a Mueller matrix [nlam][4][nmu]
// (NULL: unpolarized), with internal sources Lsrc per cell (erg/s; NULL: none), keeping the mean-intensity path lengths when jlen is given (nr*nt*nlam, internal
// length units; not with a Mueller matrix). Returns the tallies (nr*nt: fixed-point energy, entries,
// absorptions), the escape counts and Stokes Q/I, U/I tallies (nlam * 10) and the counters {packets,
// absorptions, scatterings, crossings, MRW jumps, capped, escaped, error flags}.
extern "C" void host_transport(int nr, int nt, const double* rf_cm, const double* tf, const double* rho, int nlam,
                               const double* lam_e, const double* kabs, const double* ksca, const double* g,
                               double Tstar, double Rstar, uint64_t n, uint64_t seed, int mrw, double gamma, int nmin,
                               int want_sed, int prec, int nmu, const double* mueller, const double* Lsrc,
                               uint64_t* tally,
                               uint64_t* visits, uint64_t* nabs, uint64_t* sed, uint64_t* sed_q, uint64_t* sed_u,
                               double* jlen, uint64_t* counters) {
  const Inputs in{nr, nt, nlam, rf_cm, tf, rho, lam_e, kabs, ksca, g, Tstar, Rstar, n, seed, mrw, nmin, want_sed, nmu,
                  gamma, mueller, Lsrc, 0, nullptr};
  const Outputs out{tally, visits, nabs, sed, sed_q, sed_u, counters, jlen, nullptr};
  if (prec == 32) run<float>(in, out);
  else run<double>(in, out);
}

// Replays the geometry of one packet from a recorded state (see replay_advance) on the disk, FP32 (prec 32)
// or FP64, with the kernels' step guards (1e5 crossings without an interaction). state: {ir, itheta, px, py,
// pz, ux, uy, uz, tau, xcross, max_calls}; out: {advance calls, face crossings, last result (0 ended,
// 1 crossed, 2 interaction point), error flags, ir, itheta}.
extern "C" void host_replay(int nr, int nt, const double* rf_cm, const double* tf, const double* rho, int nlam,
                            const double* lam_e, const double* kabs, const double* ksca, const double* g, double Tstar,
                            double Rstar, int prec, const double* state, int64_t* out) {
  const Inputs in{nr, nt, nlam, rf_cm, tf, rho, lam_e, kabs, ksca, g, Tstar, Rstar, 1, 1, 0, 20, 0, 0,
                  2.0, nullptr, nullptr, 0, state};
  std::vector<uint64_t> t((size_t)nr * nt), v((size_t)nr * nt), a((size_t)nr * nt), sed((size_t)nlam * kNInc),
      cnt(8);
  const Outputs o{t.data(), v.data(), a.data(), sed.data(), nullptr, nullptr, cnt.data(), nullptr, out};
  if (prec == 32) run<float>(in, o);
  else run<double>(in, o);
}

// host_transport with `lanes` packets in flight at once (run_interleaved; unpolarized, no J tally)
extern "C" void host_transport_interleaved(int nr, int nt, const double* rf_cm, const double* tf, const double* rho,
                                           int nlam, const double* lam_e, const double* kabs, const double* ksca,
                                           const double* g, double Tstar, double Rstar, uint64_t n, uint64_t seed,
                                           int mrw, double gamma, int nmin, int want_sed, int prec, uint64_t lanes,
                                           uint64_t* tally, uint64_t* visits, uint64_t* nabs, uint64_t* sed,
                                           uint64_t* counters) {
  const Inputs in{nr, nt, nlam, rf_cm, tf, rho, lam_e, kabs, ksca, g, Tstar, Rstar, n, seed, mrw, nmin, want_sed, 0,
                  gamma, nullptr, nullptr, lanes, nullptr};
  std::vector<uint64_t> q((size_t)nlam * kNInc), u((size_t)nlam * kNInc);
  const Outputs out{tally, visits, nabs, sed, q.data(), u.data(), counters, nullptr, nullptr};
  if (prec == 32) run<float>(in, out);
  else run<double>(in, out);
}
