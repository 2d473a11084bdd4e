"""Host logic of bench.py (CPU): the kernel-launch count it reports as `gpu_launches`.

Per batched ADMM iteration libselr launches the adjoint (1), the transforms of the
adjoints (2 for 2D models, 1 otherwise), the DC divide and its reduction (2), the hybrid
transforms (2 / 1), the lift (1), and for every run of consecutive lift families of one
SVT size class either the warp-per-matrix SVT (s <= 8, len <= 64: 1 kernel), or the Gram,
tridiagonal reduction, eigenvectors, three apply kernels and the FP64 re-solve of flagged
matrices (eigensolver: 7), or Jacobi and apply (2); parameter models add the copy of the
active flags (1).  The 12-coil 256x256 iteration has 15 kernels: tridiag, eigvec, Gram,
the three apply kernels, the FP64 re-solve, lift, four transforms, adjoint, DC and the
reduction.
"""
import bench


class _Desc:
    def __init__(self, model, J=12, cg_iters=30):
        self.model, self.J, self.cg_iters = model, J, cg_iters


class _Plan:
    def __init__(self, fams, desc=None):
        self._f = fams
        if desc is not None:
            self.desc = desc

    def lift_shape(self, axis):
        return self._f[axis]


def test_bench_workload_counts_fifteen_per_iteration():
    p = _Plan({"row": (256, 241, 192), "col": (256, 241, 192)})
    assert bench.kernel_launches_per_iteration(p, True, "batched") == 15
    assert bench.kernel_launches_per_iteration(p, True, "batched", svd="jacobi") == 10


def test_two_stage_reduction_adds_one_launch_per_eligible_sequence():
    # k_sb1 + k_sb2 replace k_tridiag where every order of the sequence lies in 48 .. 192
    p = _Plan({"row": (256, 241, 192), "col": (256, 241, 192)})
    assert bench.kernel_launches_per_iteration(p, True, "batched", reduction=2) == 16
    assert bench.kernel_launches_per_iteration(p, True, "batched", reduction=1) == 15
    # order 384 (outside the range) keeps the one-stage sequence; order 192 gets two-stage
    p = _Plan({"row": (256, 241, 384), "col": (256, 241, 192)})
    assert bench.kernel_launches_per_iteration(p, True, "batched", reduction=2) == 8 + 15
    # plain: one more kernel per eligible matrix (orders 32 stay one-stage)
    p = _Plan({"row": (4, 57, 48), "col": (4, 57, 32)})
    assert (bench.kernel_launches_per_iteration(p, True, "plain", reduction=2)
            == bench.kernel_launches_per_iteration(p, True, "plain") + 4)


def test_families_in_different_classes_get_their_own_sequence():
    # SHLR-V-like rows (s = 241) and a family of s = 192: two eigensolver sequences
    p = _Plan({"row": (256, 241, 384), "col": (256, 241, 192)})
    assert bench.kernel_launches_per_iteration(p, True, "batched") == 8 + 14


def test_parameter_model_small_and_eig_classes():
    # SHLR-VP: 1536 PE lifts 181x192 (eigensolver) + 36864 parameter lifts 5x32 (warp SVT)
    p = _Plan({"pe": (1536, 181, 192), "param": (36864, 5, 32)})
    assert bench.kernel_launches_per_iteration(p, False, "batched") == 1 + 1 + 2 + 1 + 1 + 7 + 1 + 1


def test_plain_mode_counts_per_matrix():
    p = _Plan({"row": (4, 57, 32), "col": (4, 57, 32)})
    # per matrix: its lift and its seven eigensolver kernels
    assert bench.kernel_launches_per_iteration(p, True, "plain") == 8 + 2 + 2 + 2 + 8 * 8


def test_spirit_models_count_the_cg_x_update_and_the_calibration():
    # SHLR-S: the pointwise divide (1 kernel) becomes the CG X-update: copy, operator
    # (4 FFTs + pixel + combine), init, 30 x (operator, update, direction update) less the
    # last direction update, finish = 8 + 8 * 30 kernels
    fams = {"row": (256, 241, 192), "col": (256, 241, 192)}
    p = _Plan(fams, _Desc("SHLR_S", J=12, cg_iters=30))
    assert bench.kernel_launches_per_iteration(p, True, "batched") == 15 - 1 + 8 + 8 * 30
    # calibration once per solve: Gram, 3 Cholesky launches (4 coils each), place, 2 FFTs, finish
    assert bench.calibration_launches(p) == 5 + 3
    assert bench.calibration_launches(_Plan(fams, _Desc("SHLR"))) == 0


def test_svd_traffic_scales_the_captured_bytes_per_matrix():
    # the full-size capture of k_tridiag + k_eigvec at order 192 covers 512 matrices
    assert abs(bench.svd_traffic([(256, 192), (256, 192)]) - (75.94e6 + 18.22e6 + 77.59e6 + 0.06e6)) < 1.0
    assert bench.svd_traffic([(256, 241)]) is None
    assert bench.svd_traffic([]) is None
