// Continuous-batching request server for ASCC solves on one GPU.
//
// Requests (one molecule, one or more states) are queued as they arrive;
// worker threads, each with its own CUDA stream, admit the oldest request
// whose device footprint fits in the memory budget next to the requests
// already running, build its bare integrals once, solve its states (sharing
// the molecule) and release the memory.  Work of concurrently admitted
// requests overlaps on the device through the workers' streams.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>

#include "engine.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int o, v, naux;
  std::vector<double> eps, B;
  std::vector<ascc_excitation> states;
  double t_arrival;
  size_t footprint;
};

}  // namespace

struct ascc_server {
  ascc_server(size_t budget, int workers, const ascc::Options& opt, const ascc_options& raw,
              int device)
      : budget_(budget), nworkers_(workers), opt_(opt), raw_(raw), device_(device),
        t0_(Clock::now()) {}
  const ascc_options& raw_options() const { return raw_; }
  ~ascc_server() { stop(); }

  double now() const { return std::chrono::duration<double>(Clock::now() - t0_).count(); }

  int64_t submit(Request r) {
    std::lock_guard<std::mutex> lk(mu_);
    r.id = next_id_++;
    r.t_arrival = now();
    queue_.push_back(std::move(r));
    cv_.notify_all();
    return queue_.back().id;
  }

  void start() {
    std::lock_guard<std::mutex> lk(mu_);
    if (!threads_.empty()) return;
    stopping_ = false;
    for (int w = 0; w < nworkers_; ++w) threads_.emplace_back([this, w] { worker(w); });
  }

  // Blocks until every submitted request has finished.
  void drain() {
    std::unique_lock<std::mutex> lk(mu_);
    cv_.wait(lk, [&] { return queue_.empty() && running_ == 0; });
  }

  void stop() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stopping_ = true;
      cv_.notify_all();
    }
    for (auto& t : threads_) t.join();
    threads_.clear();
  }

  size_t budget() const { return budget_; }
  std::vector<ascc_serve_result> results() {
    std::lock_guard<std::mutex> lk(mu_);
    return results_;
  }
  std::string first_error() {
    std::lock_guard<std::mutex> lk(mu_);
    return error_;
  }

 private:
  void worker(int w) {
    cudaSetDevice(device_);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    while (true) {
      Request r;
      {
        std::unique_lock<std::mutex> lk(mu_);
        // admission: the oldest queued request whose footprint fits beside the
        // running ones (a large request at the head does not hold back smaller
        // ones behind it); every queued request fits the budget on its own
        auto pick = [&]() -> std::deque<Request>::iterator {
          for (auto it = queue_.begin(); it != queue_.end(); ++it)
            if (in_use_ + it->footprint <= budget_) return it;
          return queue_.end();
        };
        cv_.wait(lk, [&] { return stopping_ || pick() != queue_.end(); });
        auto it = pick();
        if (it == queue_.end()) break;  // stopping, nothing admissible
        r = std::move(*it);
        queue_.erase(it);
        in_use_ += r.footprint;
        ++running_;
      }
      const double t_start = now();
      std::vector<ascc_serve_result> out;
      try {
        const int build_level = opt_.precision == ASCC_MIXED_BF16 ? 3 : 0;
        auto mol = std::make_shared<ascc::Molecule>(r.o, r.v, r.naux, r.eps.data(), r.B.data(),
                                                    false, s, build_level);
        r.B.clear();
        r.B.shrink_to_fit();
        for (size_t k = 0; k < r.states.size(); ++k) {
          const ascc_excitation& e = r.states[k];
          ascc::Options o = opt_;
          int hole = -1, particle = -1;
          if (e.n_csf == 1) {
            hole = e.hole;
            particle = e.particle;
          } else {
            // the ground state takes the primary labels of the request's first excitation
            for (const auto& x : r.states)
              if (x.n_csf == 1) {
                o.pl_hole = x.hole;
                o.pl_particle = x.particle;
                break;
              }
          }
          double beta = e.beta, xsign = 1.0;
          if (e.n_csf == 1) {
            xsign = e.ansatz == 1 ? -1.0 : 1.0;
            if (beta == 0.0) beta = e.ansatz == 1 ? 1.0 / (1.0 - e.alpha) : 1.0 / (1.0 + e.alpha);
          }
          ascc_result res{};
          {
            ascc::State st(mol, hole, particle, beta, o, s, xsign);
            st.solve(&res);
          }
          if (o.precision == ASCC_MIXED_BF16 && res.status == ASCC_ERR_NOT_CONVERGED) {
            // a mixed solve that did not converge is solved again on the
            // FP64-class path (the molecule holds its digit planes), so that a
            // state the FP64-class iteration converges is not lost to the
            // low-precision phase; the result counts both solves' iterations
            ascc::Options o2 = o;
            o2.precision = ASCC_FP64_TC;
            ascc_result res2{};
            ascc::State st2(mol, hole, particle, beta, o2, s, xsign);
            st2.solve(&res2);
            res2.iterations += res.iterations;
            res = res2;
          }
          ascc_serve_result sr{};
          sr.request_id = r.id;
          sr.state_index = (int32_t)k;
          sr.status = res.status;
          sr.energy = res.energy;
          sr.iterations = res.iterations;
          sr.worker = w;
          sr.t_arrival = r.t_arrival;
          sr.t_start = t_start;
          sr.t_end = now();
          out.push_back(sr);
        }
      } catch (const std::exception& ex) {
        std::lock_guard<std::mutex> lk(mu_);
        if (error_.empty()) error_ = ex.what();
        ascc_serve_result sr{};
        sr.request_id = r.id;
        sr.state_index = -1;
        sr.status = ASCC_ERR_CUDA;
        if (auto* ae = dynamic_cast<const ascc::Error*>(&ex)) sr.status = ae->status;
        sr.t_arrival = r.t_arrival;
        sr.t_start = t_start;
        sr.t_end = now();
        out.push_back(sr);
      }
      cudaStreamSynchronize(s);
      {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto& x : out) results_.push_back(x);
        in_use_ -= r.footprint;
        --running_;
        cv_.notify_all();
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }

  size_t budget_;
  int nworkers_;
  ascc::Options opt_;
  ascc_options raw_;
  int device_;
  Clock::time_point t0_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Request> queue_;
  std::vector<std::thread> threads_;
  std::vector<ascc_serve_result> results_;
  std::string error_;
  size_t in_use_ = 0;
  int running_ = 0;
  int64_t next_id_ = 0;
  bool stopping_ = false;
};

namespace {
ascc::Options options_from(const ascc_options* o) {
  ascc::Options r;
  if (!o) return r;
  r.precision = o->precision;
  r.linearize = o->linearize;
  r.triples = o->triples;
  r.pl_hole = o->pl_hole;
  r.pl_particle = o->pl_particle;
  r.r_tol = o->r_tol;
  r.e_tol = o->e_tol;
  r.max_iter = o->max_iter;
  r.diis_dim = o->diis_dim;
  r.diis_start = o->diis_start;
  r.polish_iter = o->polish_iter;
  r.polish_tol = o->polish_tol;
  r.ladder_stream = o->ladder_stream;
  return r;
}

template <class F>
ascc_status guarded(F&& f) {
  try {
    return f();
  } catch (const ascc::Error& e) {
    ascc::record_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    ascc::record_error(e.what());
    return ASCC_ERR_INVALID;
  }
}
}  // namespace

extern "C" {

ascc_status ascc_server_create(ascc_server** out, size_t memory_budget, int32_t max_active,
                               const ascc_options* opt) {
  if (out) *out = nullptr;
  return guarded([&]() -> ascc_status {
    ASCC_REQUIRE(out && max_active >= 1 && max_active <= 64, "max_active in 1..64");
    int dev = 0;
    ASCC_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    ASCC_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;
    ASCC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    ascc_options raw;
    if (opt) raw = *opt; else ascc_default_options(&raw);
    auto* s = new ascc_server(memory_budget, max_active, options_from(&raw), raw, dev);
    s->start();
    *out = s;
    return ASCC_OK;
  });
}

ascc_status ascc_server_submit(ascc_server* srv, int32_t o, int32_t v, int32_t naux,
                               const double* eps, const double* B, int32_t n_states,
                               const ascc_excitation* states, int64_t* request_id) {
  return guarded([&]() -> ascc_status {
    ASCC_REQUIRE(srv && eps && B && states && n_states >= 1, "null argument");
    ASCC_REQUIRE(o >= 1 && v >= 1 && naux >= 1, "sizes must be positive");
    for (int k = 0; k < n_states; ++k) {
      const auto& e = states[k];
      ASCC_REQUIRE(e.n_csf == 0 || (e.n_csf == 1 && e.hole >= 0 && e.hole < o &&
                                    e.particle >= 0 && e.particle < v),
                   "bad excitation");
    }
    Request r;
    r.o = o;
    r.v = v;
    r.naux = naux;
    const int n = o + v;
    r.eps.assign(eps, eps + n);
    r.B.assign(B, B + (size_t)naux * n * n);
    r.states.assign(states, states + n_states);
    r.footprint = ascc_footprint_bytes(o, v, naux, &srv->raw_options());
    if (r.footprint > srv->budget())
      throw ascc::Error(ASCC_ERR_OOM, "request needs " + std::to_string(r.footprint) +
                                          " device bytes, more than the server's budget of " +
                                          std::to_string(srv->budget()));
    const int64_t id = srv->submit(std::move(r));
    if (request_id) *request_id = id;
    return ASCC_OK;
  });
}

ascc_status ascc_server_drain(ascc_server* srv) {
  return guarded([&]() -> ascc_status {
    ASCC_REQUIRE(srv, "null argument");
    srv->drain();
    return ASCC_OK;
  });
}

int64_t ascc_server_result_count(ascc_server* srv) {
  return srv ? (int64_t)srv->results().size() : 0;
}

ascc_status ascc_server_results(ascc_server* srv, ascc_serve_result* out, int64_t capacity) {
  return guarded([&]() -> ascc_status {
    ASCC_REQUIRE(srv && out, "null argument");
    auto r = srv->results();
    ASCC_REQUIRE((int64_t)r.size() <= capacity, "result buffer too small");
    if (!r.empty()) std::memcpy(out, r.data(), r.size() * sizeof(ascc_serve_result));
    return ASCC_OK;
  });
}

void ascc_server_destroy(ascc_server* srv) { delete srv; }

}  // extern "C"
