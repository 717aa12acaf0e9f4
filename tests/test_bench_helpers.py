"""Host-side helpers of bench.py (no GPU).

- roofline.traffic comes from a committed ncu summary only while the stage
  kernel sources hash to the value recorded beside it; the hash covers the
  code, not its comments or white space;
- the dominant kernel is the (family, lines per CTA) most timed plans chose;
- the FP32-issue roofline counts the double-float radix-pass arithmetic:
  16 operations per complex addition, 32 per twiddle product, radix 2 / 4 / 8
  butterflies at 16 / 32 / 54 per point;
- the oracle baseline never plans more threads than host memory holds.
"""
import os

import bench


def test_profiled_traffic_follows_the_source_hash(tmp_path):
    h = bench.stage_source_hash()
    assert len(h) == 16
    summary = tmp_path / "summary.md"
    summary.write_text("text\n\n    source_hash: %s\n    dram_bytes_per_point G8: 29.5\n" % h)
    assert bench.profiled_traffic(h, "warp", 8, 512, str(summary)) == 29.5
    assert bench.profiled_traffic("0" * 16, "warp", 8, 512, str(summary)) is None     # stale hash: no figure
    assert bench.profiled_traffic(h, "warp", 5, 512, str(summary)) is None            # no such capture
    assert bench.profiled_traffic(h, "warp", 8, 512, str(tmp_path / "absent.md")) is None


def test_source_hash_ignores_comments_and_white_space():
    a = "int f(int x) {  // twice x\n    return 2 * x; /* the\n  value */\n}\n"
    b = "int f(int x) {\n  return 2 * x;\n}"
    assert bench.source_code_only(a) == bench.source_code_only(b) == "int f(int x) { return 2 * x; }"
    assert bench.source_code_only(a) != bench.source_code_only(b.replace("2", "3"))


def test_profiled_traffic_of_the_committed_summaries():
    for n in (256, 512):
        path = os.path.join(os.path.dirname(bench.__file__), "profiles", "fft_warp_kernel_df_n%d.md" % n)
        with open(path) as fh:
            h = [ln.split(":", 1)[1].strip() for ln in fh if ln.strip().startswith("source_hash:")][0]
        for G in (4, 8):
            v = bench.profiled_traffic(h, "warp", G, n)
            assert v is not None and 28.0 < v < 32.0, (n, G, v)     # about 2 x 16 bytes per point


def test_dominant_kernel():
    chosen = {16: {"kernel": 0, "lines_per_cta": 8}, 64: {"kernel": 0, "lines_per_cta": 8},
              256: {"kernel": 2, "lines_per_cta": 4}}
    assert bench.dominant_kernel(chosen) == ("warp", 8)
    chosen = {16: {"kernel": 2, "lines_per_cta": 4}, 64: {"kernel": 2, "lines_per_cta": 4},
              256: {"kernel": 0, "lines_per_cta": 8}}
    assert bench.dominant_kernel(chosen) == ("tile", 4)


def test_double_float_operation_count():
    add, mul = 16.0, 32.0
    radix4 = 8 * add / 4                               # two levels of 2 complex additions per pair
    radix8 = (2 * 8 * add + 2 * (add + 8) + 8 * add) / 8  # two radix-4 halves, two (1 -+ i)/sqrt2 factors, 8 additions
    assert radix4 == 32 and radix8 == 54
    assert bench.df_ops_per_point(8) == radix8
    assert bench.df_ops_per_point(64) == radix8 + radix8 + mul * 7 / 8
    assert bench.df_ops_per_point(256) == radix4 + 2 * (radix8 + mul * 7 / 8) == 196
    assert bench.df_ops_per_point(512) == radix8 + 2 * (radix8 + mul * 7 / 8)
    assert bench.df_ops_per_point(32) == radix4 + radix8 + mul * 7 / 8


def test_host_threads_respects_memory():
    cores = len(os.sched_getaffinity(0))
    assert 1 <= bench.host_threads(1) <= cores
    assert bench.host_threads(1 << 60) == 1                     # nothing fits: still one thread
