"""Plain-C FP64 oracle of the calorimeter hit path: test infrastructure only."""
