"""Host-side accounting of bench.py (no GPU): the padded sizes the kernels execute
over, the kernel names a plan launches, and the executed tensor-core flops of the two
passes, checked against hand counts for the L = 96, K = 3, N = 5e4 workload."""
import bench


class P:  # the fields of a synthetic problem that the accounting reads
    L, K, N = 96, 3, 50_000

    @property
    def l(self):
        return self.L // self.K


def test_padded_sizes():
    Npad, Spad, ldk, nch = bench.padded(P())
    assert (Npad, Spad, ldk, nch) == (50_048, 9216, 1024, 4)


def test_kernel_names_follow_the_plan():
    plan = {"p2_form": "ring", "p1_shift_tile": 256}
    assert bench.kernel_names("bf16x3", plan, 32) == ("k_p1_tc<3,256>", "k_p2c_tc<3>")
    plan = {"p2_form": "per_chunk_comp", "p1_shift_tile": 128}
    assert bench.kernel_names("bf16x3", plan, 32) == ("k_p1_tc<3,128>", "k_p2_tc<3,true>")
    assert bench.kernel_names("bf16", {"p2_form": "interleaved"}, 32)[1] == "k_p2i_tc<1>"
    assert bench.kernel_names("fp32", {}, 32) == ("k_p1_f32", "k_p2_f32")
    assert bench.kernel_names("fft32", {}, 16) == ("k_fft_p1<16>", "k_fft_p2<16>")


def test_executed_tensor_flops():
    # pass 1: 3 MMAs x 2 flops x 50048 observations x 9216 shifts x 1024 pixels
    p1, p2 = bench.tc_executed_flops(P(), "bf16x3", {"p2_chunk_groups": 1, "p2_form": "ring"})
    assert p1 == 3 * 2.0 * 50_048 * 9216 * 1024
    # pass 2: the logits once (one chunk group) + Z' over 4 chunks of 256 pixels
    assert p2 == 3 * 2.0 * 9216 * 50_048 * 1024 + 2.0 * 9216 * 50_048 * 1024
    # per-chunk kernel: the logits once per chunk; the compensated M-step triples Z'
    _, q2 = bench.tc_executed_flops(P(), "bf16x3", {"p2_chunk_groups": 4,
                                                    "p2_form": "per_chunk_comp"})
    assert q2 == 4 * 3 * 2.0 * 9216 * 50_048 * 1024 + 3 * 2.0 * 9216 * 50_048 * 1024
    _, b2 = bench.tc_executed_flops(P(), "bf16", {"p2_chunk_groups": 1, "p2_form": "ring"})
    assert b2 == 2.0 * 9216 * 50_048 * 1024 + 2.0 * 9216 * 50_048 * 1024


def test_fp32_peak_and_job_throughput():
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.54784) < 1e-9
    assert bench.job_throughput(100.0, 10, 2, 500.0) == 2 * 100.0 * 10 / 0.5
