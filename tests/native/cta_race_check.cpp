// Race check of the cooperative 3D cell routines that the CUDA kernels run
// (cell residual, cell Jacobian, Vanka set-up and apply).
//
// Each routine is written once for a thread group (fsi_cta.h). The CPU tests
// run it as one host thread, where a missing barrier cannot show. Here it runs
// on nt real host threads, each taking the work items of one CUDA thread
// (e = tid, tid + nt, ...), with a std::barrier for every sync(). Built with
// ThreadSanitizer, any access that a barrier does not order against a
// conflicting one is reported; the result must also equal the one-thread run
// bit for bit. Exit code 0 when every case agrees, 1 otherwise.
#include <barrier>
#include <cstdio>
#include <cstring>
#include <functional>
#include <random>
#include <thread>
#include <vector>

#include "../../paper_1907_01252_gb300/csrc/fsi_element3d.cuh"
#include "../../paper_1907_01252_gb300/csrc/fsi_mesh3d.h"
#include "../../paper_1907_01252_gb300/csrc/fsi_vanka3.h"

namespace {

struct ThreadCta {
  int tid, nt;
  std::barrier<>* bar;
  void sync() const { bar->arrive_and_wait(); }
};

void run_threads(int nt, const std::function<void(const ThreadCta&)>& body) {
  std::barrier<> bar(nt);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back([&, t] { body(ThreadCta{t, nt, &bar}); });
  for (auto& x : th) x.join();
}

int failures = 0;

template <typename T>
void expect_equal(const char* what, const std::vector<T>& a, const std::vector<T>& b) {
  if (a.size() != b.size() || std::memcmp(a.data(), b.data(), a.size() * sizeof(T)) != 0) {
    std::printf("MISMATCH %s\n", what);
    ++failures;
  } else {
    std::printf("ok %s\n", what);
  }
}

void random_cell_state(std::mt19937_64& g, std::vector<double>& U) {
  std::uniform_real_distribution<double> d(-1.0, 1.0);
  for (int l = 0; l < 27; ++l) {
    for (int c = 0; c < 3; ++c) U[l * 7 + c] = d(g);
    for (int c = 3; c < 6; ++c) U[l * 7 + c] = 2e-3 * d(g);
    U[l * 7 + 6] = 100.0 * d(g);
  }
}

void check_cell_routines(int nt) {
  fsi3::Tables3 T;
  fsi3::build_tables3(T);
  const fsi3::Phys3 P{1000.0, 1e-3, 1000.0, 5e5, 2e6};
  const double h[3] = {0.05, 0.0525, 0.05};
  std::mt19937_64 g(1907);
  std::vector<double> Ue(189), Uo(189);
  for (int kind = 0; kind < 3; ++kind) {   // fluid, solid, outflow fluid cell
    const bool solid = kind == 1, outflow = kind == 2;
    random_cell_state(g, Ue);
    random_cell_state(g, Uo);
    const double k = 0.01, theta = 0.51, alpha = 3e-7;
    // residual
    std::vector<double> sh1(fsi3::CR3_TOTAL, -1.0), shn(fsi3::CR3_TOTAL, -2.0), R1(189, -7.0), Rn(189, -8.0);
    std::copy(Ue.begin(), Ue.end(), sh1.begin() + fsi3::CR3_UE);
    std::copy(Uo.begin(), Uo.end(), sh1.begin() + fsi3::CR3_UE + 189);
    std::copy(sh1.begin() + fsi3::CR3_UE, sh1.begin() + fsi3::CR3_UE + 378, shn.begin() + fsi3::CR3_UE);
    fsi3::cell_residual3_cta(fsi3::HostCta{}, P, T, h, solid, outflow, k, theta, alpha, sh1.data(), R1.data());
    run_threads(nt, [&](const ThreadCta& c) {
      fsi3::cell_residual3_cta(c, P, T, h, solid, outflow, k, theta, alpha, shn.data(), Rn.data());
    });
    char name[64];
    std::snprintf(name, sizeof name, "cell_residual3_cta kind %d", kind);
    expect_equal(name, R1, Rn);
    // Jacobian
    std::vector<double> sj1(fsi3::CJ3_TOTAL, -1.0), sjn(fsi3::CJ3_TOTAL, -2.0);
    std::vector<double> K1(189 * 189, -7.0), Kn(189 * 189, -8.0);
    std::copy(Ue.begin(), Ue.end(), sj1.begin() + fsi3::CJ3_UE);
    std::copy(Uo.begin(), Uo.end(), sj1.begin() + fsi3::CJ3_UE + 189);
    std::copy(sj1.begin() + fsi3::CJ3_UE, sj1.begin() + fsi3::CJ3_UE + 378, sjn.begin() + fsi3::CJ3_UE);
    fsi3::cell_jacobian3_cta(fsi3::HostCta{}, P, T, h, solid, outflow, k, theta, alpha, sj1.data(), K1.data());
    run_threads(nt, [&](const ThreadCta& c) {
      fsi3::cell_jacobian3_cta(c, P, T, h, solid, outflow, k, theta, alpha, sjn.data(), Kn.data());
    });
    std::snprintf(name, sizeof name, "cell_jacobian3_cta kind %d", kind);
    expect_equal(name, K1, Kn);
  }
}

template <typename TV>
void check_vanka(int nt) {
  // 5 x 2 x 3 cells of the channel with the plate (solid, coupled and decoupled fluid cells)
  const double xb[4] = {0.0, 0.4, 0.45, 1.5}, yb[3] = {0.0, 0.2, 0.41}, zb[4] = {0.0, 0.055, 0.355, 0.41};
  const int nxs[3] = {1, 1, 3}, nys[2] = {1, 1}, nzs[3] = {1, 1, 1};
  const double box[6] = {0.4, 0.45, 0.0, 0.2, 0.055, 0.355};
  fsi3::HostMesh3 m;
  fsi3::build_mesh3(m, fsi3::axis_vertices3(xb, nxs, 3), fsi3::axis_vertices3(yb, nys, 2),
                    fsi3::axis_vertices3(zb, nzs, 3), box);
  const fsi3::Mesh3View v{m.nnx, m.nny, m.nnz, m.n_nodes, m.n_cells, m.yn.data(), m.zn.data(),
                          m.cell_flags.data(), m.node_flags.data(), m.node_cells.data(), m.y0, m.y1, m.z0, m.z1,
                          m.blk_row.data(), m.colidx.data(), m.blk_src.data(), m.cell_blk.data()};
  // a random block matrix with a dominant diagonal (every local matrix is regular), and the
  // structure of decoupled cells: their displacement rows see only their own component
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> d(-1.0, 1.0);
  std::vector<TV> A((size_t)m.nnzb * 49);
  for (int b = 0; b < m.nnzb; ++b) {
    const bool diag = m.blk_row[b] == m.colidx[b];
    const bool coupled = m.node_flags[m.blk_row[b]] & fsi3::N3_IN_SOLID;
    for (int r = 0; r < 7; ++r)
      for (int c = 0; c < 7; ++c) {
        double x = 0.1 * d(g);
        if (!coupled && r >= 3 && r < 6 && c != r) x = 0.0;
        if (diag && r == c) x += 60.0;
        A[(size_t)b * 49 + r * 7 + c] = (TV)x;
      }
  }
  int cells_done = 0, decoupled = 0;
  for (int cell = 0; cell < m.n_cells; ++cell) {
    std::vector<TV> sh1(fsi3::VK3_SH_T), shn(fsi3::VK3_SH_T), inv1(fsi3::VK3_SIZE), invn(fsi3::VK3_SIZE);
    std::vector<int> ish1(fsi3::VK3_SH_I), ishn(fsi3::VK3_SH_I);
    const bool ok1 = fsi3::vk3_setup_cell(fsi3::HostCta{}, v, A.data(), cell, sh1.data(), ish1.data(), inv1.data());
    std::vector<int> okn(nt, 0);
    run_threads(nt, [&](const ThreadCta& c) {
      okn[c.tid] = fsi3::vk3_setup_cell(c, v, A.data(), cell, shn.data(), ishn.data(), invn.data());
    });
    for (int t = 0; t < nt; ++t)
      if (okn[t] != (int)ok1) {
        std::printf("MISMATCH vk3_setup_cell status cell %d\n", cell);
        ++failures;
      }
    char name[64];
    std::snprintf(name, sizeof name, "vk3_setup_cell cell %d", cell);
    expect_equal(name, inv1, invn);
    const bool dec = (m.cell_flags[cell] & fsi3::C3_U_DECOUPLED) != 0;
    std::vector<TV> r(189), ap1(fsi3::VK3_AP_T), apn(fsi3::VK3_AP_T), z1(189, TV(-7)), zn(189, TV(-8));
    for (auto& x : r) x = (TV)d(g);
    fsi3::vk3_apply_cell(fsi3::HostCta{}, dec, inv1.data(), r.data(), ap1.data(), z1.data());
    run_threads(nt, [&](const ThreadCta& c) { fsi3::vk3_apply_cell(c, dec, invn.data(), r.data(), apn.data(), zn.data()); });
    std::snprintf(name, sizeof name, "vk3_apply_cell cell %d", cell);
    expect_equal(name, z1, zn);
    ++cells_done;
    decoupled += dec;
  }
  std::printf("vanka: %d cells, %d decoupled\n", cells_done, decoupled);
}

}  // namespace

int main(int argc, char** argv) {
  const int nt = argc > 1 ? std::atoi(argv[1]) : 8;
  check_cell_routines(nt);
  check_vanka<double>(nt);
  check_vanka<float>(nt);
  std::printf("%s\n", failures ? "FAILED" : "PASSED");
  return failures ? 1 : 0;
}
