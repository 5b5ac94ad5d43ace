"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws data (networks, scenario trees, forecasts, prices); it
contains none of the solver's arithmetic, so both the CPU oracle and the CUDA
path can consume the same inputs without sharing any solver code.
"""
from .networks import demand_forecast, make_network, make_tiny_network, node_deviations  # noqa: F401
from .problems import (assemble, barcelona, batch_instances, custom, forest, forest_members,  # noqa: F401
                       general_dynamics, large, random_instance, tiny)
from .trees import (make_tree, random_tree, stages_of, tree_from_fanouts, tree_from_fanouts_dict,  # noqa: F401
                    uniform_scenario_probabilities)
