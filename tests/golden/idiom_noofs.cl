__kernel void idiom(__global int *data)
{
    data[(get_global_id(0) - get_global_offset(0))] = (int)(get_global_id(0) - get_global_offset(0));
}
