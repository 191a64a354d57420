"""Host helpers of the benchmark (no GPU): the CPU list of the GPU's NUMA
node that the end-to-end section runs on."""
import os

import bench


def test_cpu_lists_parse_ranges_and_singletons():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("0-0,2-2") == {0, 2}
    assert bench.parse_cpulist("") == set()


def test_local_cpus_are_none_or_cpus_this_process_may_use():
    # without nvidia-smi or the sysfs entry the section stays unbound
    cpus = bench.gpu_local_cpus(0)
    assert cpus is None or (cpus and cpus <= os.sched_getaffinity(0))
