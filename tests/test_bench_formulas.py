"""The algorithmic work that bench.py divides by time (the roofline numerators), checked against figures
worked out independently of it: the per-step flops and compulsory bytes printed for the benchmark
workloads (F_gemm = 16 nb nr nv nf, F_fft = 5 nfft log2(nfft) (nr nv + nb nv) with nfft the smallest
2^a 3^b 5^c >= 2 nt - 1, bytes = X read + write, the gathered kernel spectra, the batch rows of U_obs,
and the G round trip with reciprocity), to the digits they are printed with, and the fused update
kernel's algorithmic and staged bytes per launch worked by hand."""
import pytest

import bench

# workload: (nt, nr, nv, nb, reciprocity) -> (F_gemm GF, F_fft GF, compulsory MB)
PRINTED = {
    (512, 201, 201, 16, True): (5.31, 2.23, 351),
    (512, 256, 256, 16, True): (8.61, 3.57, 562),
    (1024, 301, 301, 32, False): (47.5, 11.3, 861),
    (1024, 301, 301, 64, False): (95.1, 12.4, 979),
    (1500, 1200, 1200, 32, False): (1107, 256, 18.0e3),
}


@pytest.mark.parametrize("shape", list(PRINTED), ids=lambda s: "x".join(map(str, s)))
def test_step_work_matches_printed_figures(shape):
    nt, nr, nv, nb, recip = shape
    f_gemm, f_fft, mb = PRINTED[shape]
    nfft = bench.nfft_for(nt)
    nf = nfft // 2 + 1
    gemm = 16.0 * nb * nr * nv * nf
    total = bench.step_flops(nt, nr, nv, nb)
    assert gemm / 1e9 == pytest.approx(f_gemm, rel=6e-3)
    assert (total - gemm) / 1e9 == pytest.approx(f_fft, rel=6e-3)
    assert bench.step_bytes_compulsory(nt, nr, nv, nb, recip) / 1e6 == pytest.approx(mb, rel=6e-3)


def test_fft_length_is_the_smallest_5_smooth_at_or_above_2nt_minus_1():
    # 1080 = 2^3 3^3 5 (1025 .. 1079 all have a prime factor above 5); 3000 = 2^3 3 5^3
    assert [bench.nfft_for(nt) for nt in (1, 128, 512, 513, 1024, 1500)] == [1, 256, 1024, 1080, 2048, 3000]


def test_update_bytes_per_launch_by_hand():
    # nt 512, 201 x 201: read and write the model (512 x 4 bytes each) per model trace; the staged pipeline
    # adds the gradient spectra read and the model spectra written (513 bins x 8 bytes each)
    w = bench.kernel_work("update", 512, 201, 201, 16)
    assert w["bytes"] == 201 * 201 * 512 * 4 * 2 == 165482496
    assert w["staged"] == 201 * 201 * 513 * 8 * 2
    assert w["flops"] == 2 * 2.5 * 1024 * 10 * 201 * 201


def test_symmetric_model_work_by_hand():
    # nt 512, 201 x 201 with reciprocity and a symmetric model: 201 * 202 / 2 = 20301 distinct traces carry the
    # model FFTs; the model is read on them and written whole; the symmetric gradient is formed in the adjoint
    # product, so there is no gradient round trip
    nt, n, nb = 512, 201, 16
    up = 201 * 202 // 2
    assert bench.model_traces(n, n, True) == up == 20301
    fg, ff = bench.step_work(nt, n, n, nb, sym=True)
    assert fg == 16.0 * nb * n * n * 513
    assert ff == 2 * 2.5 * 1024 * 10 * (up + nb * n)
    assert bench.step_bytes_compulsory(nt, n, n, nb, True, sym=True) == (up + n * n) * nt * 4 + 513 * nb * n * 8 + nb * n * nt * 4
    w = bench.kernel_work("update", nt, n, n, nb, sym=True)
    assert w["bytes"] == (up + n * n) * nt * 4
    assert w["flops"] == 2 * 2.5 * 1024 * 10 * up
    assert w["staged"] == 2 * up * 513 * 8
    # without the flag nothing changes
    assert bench.step_work(nt, n, n, nb) == (16.0 * nb * n * n * 513, 2 * 2.5 * 1024 * 10 * (n * n + nb * n))
